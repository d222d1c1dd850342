"""GPU vs oracle parity of the Gaussian positional encoding (Eq. (1)) and the MLP spatial query
(Section II-C), for the tcgen05 tensor-core kernel and the SIMT kernel.

The material is an argmax over float32 scores accumulated in a different order than the
oracle's FP64 sums, so it is compared exactly wherever the oracle's top-2 margin exceeds twice
the oracle's guard band (the bound on how far bfloat16 re-rounding of the hidden activations
can move a score); inside the band the GPU's choice must be one of the scores within the band
of the maximum.  Weights (sigmoid of output 5) within a quarter of the band."""
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


def decode_gpu(vs, genomes, B, dims, kernel):
    import torch
    P = genomes.shape[0]
    sim = vs.Simulator(PHYS, mlp_kernel=kernel)
    sim.set_population(np.tile(np.asarray(dims, np.int32), (P, 1)), torch.from_numpy(genomes).cuda(),
                       vs.MODE_MLP, B=torch.from_numpy(B).cuda())
    vox = sim.voxels()
    return sim, vox


def check_decode(orc, genomes, B, dims, vox, max_band_frac=0.15):
    Q = int(np.prod(dims))
    banded = 0
    for g in range(genomes.shape[0]):
        mat, w, logits, guard = orc.mlp_query(dims, B, genomes[g])
        got = vox["decoded"][g * Q:(g + 1) * Q]
        wg = vox["w"][g * Q:(g + 1) * Q]
        scores = logits[:, :5]
        top = np.sort(scores, axis=1)
        sure = (top[:, -1] - top[:, -2]) > 2 * guard
        assert np.array_equal(got[sure], mat[sure]), g
        near = scores >= (top[:, -1:] - 2 * guard[:, None])
        assert np.all(near[~sure, got[~sure].astype(int)]), g
        banded += int((~sure).sum())
        assert np.all(np.abs(wg - w) <= 0.25 * guard + 1e-6), g
    assert banded <= max_band_frac * genomes.shape[0] * Q


@pytest.mark.parametrize("kernel", [0, 1])
def test_mlp_population_8cube(vs, orc, kernel):
    rng = np.random.default_rng(50)
    genomes, B = W.mlp_genomes(rng, 48), W.pe_matrix(rng)
    sim, vox = decode_gpu(vs, genomes, B, (8, 8, 8), kernel)
    check_decode(orc, genomes, B, (8, 8, 8), vox)
    sim.close()


@pytest.mark.parametrize("dims", [(1, 1, 1), (5, 7, 3), (10, 10, 10), (16, 4, 2)])
def test_mlp_ragged_query_counts(vs, orc, dims):
    """Query counts that leave a partial 128-row tile (and fewer rows than one tile)."""
    rng = np.random.default_rng(51)
    genomes, B = W.mlp_genomes(rng, 5), W.pe_matrix(rng)
    sim, vox = decode_gpu(vs, genomes, B, dims, 0)
    check_decode(orc, genomes, B, dims, vox)
    sim.close()


def test_mlp_more_genomes_than_sms(vs, orc):
    """Persistent CTAs: several genomes per CTA (more genomes than SMs)."""
    rng = np.random.default_rng(52)
    genomes, B = W.mlp_genomes(rng, 400), W.pe_matrix(rng)
    sim, vox = decode_gpu(vs, genomes, B, (4, 4, 4), 0)
    check_decode(orc, genomes[::37], B, (4, 4, 4),
                 {k: np.concatenate([v[g * 64:(g + 1) * 64] for g in range(0, 400, 37)]) for k, v in vox.items()})
    sim.close()


def test_mlp_zero_weights_tie_to_lowest(vs, orc):
    g = np.zeros((2, W.GENOME_LEN), np.float32)
    g[:, 20992:20998] = [0.25, 0.25, 0.25, 0.25, 0.25, 0.0]
    g[1, 20992 + 2] = 0.5
    sim, vox = decode_gpu(vs, g, W.pe_matrix(np.random.default_rng(0)), (3, 3, 3), 0)
    assert np.all(vox["decoded"][:27] == 0) and np.all(vox["decoded"][27:] == 2)
    assert np.allclose(vox["w"], 0.5)
    sim.close()


def test_tensor_and_simt_kernels_agree(vs):
    rng = np.random.default_rng(53)
    genomes, B = W.mlp_genomes(rng, 64), W.pe_matrix(rng)
    s0, v0 = decode_gpu(vs, genomes, B, (8, 8, 8), 0)
    s1, v1 = decode_gpu(vs, genomes, B, (8, 8, 8), 1)
    assert (v0["decoded"] != v1["decoded"]).mean() < 1e-3
    assert np.abs(v0["w"] - v1["w"]).max() < 1e-3
    s0.close(); s1.close()


def test_mlp_decode_then_simulate(vs, orc):
    """End to end: MLP decode on the GPU, 1000 steps, fitness; the oracle decodes and simulates
    on its own.  Robots whose decoded grids differ (a guarded near-tie) are excluded and
    counted."""
    import torch
    rng = np.random.default_rng(54)
    P = 24
    genomes, B = W.mlp_genomes(rng, P), W.pe_matrix(rng)
    sim = vs.Simulator(PHYS)
    sim.set_population(np.tile(np.int32([8, 8, 8]), (P, 1)), torch.from_numpy(genomes).cuda(),
                       vs.MODE_MLP, B=torch.from_numpy(B).cuda())
    vox = sim.voxels()
    sim.step(1000)
    f = sim.fitness()
    x, _, off = sim.state()
    sim.close()
    keep, mats, ws = [], [], []
    for g in range(P):
        mat, w, _, _ = orc.mlp_query((8, 8, 8), B, genomes[g])
        if np.array_equal(mat, vox["decoded"][g * 512:(g + 1) * 512]):
            keep.append(g)
        mats.append(mat.reshape(8, 8, 8)); ws.append(w)
    assert len(keep) >= P - 2
    pop = W.make_population([(8, 8, 8)] * len(keep), [mats[g] for g in keep])
    w = np.concatenate([ws[g] for g in keep])
    kappa = np.asarray(PHYS.k_mat)[pop.mats]
    phi = np.asarray(PHYS.phase_mat)[pop.mats]
    ref = orc.run_population(pop, PHYS, 1000, w=w, kappa=kappa, phi=phi, want_x=True)
    xs = np.concatenate([x[off[g]:off[g + 1]] for g in keep])
    offs = np.concatenate([[0], np.cumsum([off[g + 1] - off[g] for g in keep])])
    check_population(orc, pop, PHYS, 1000, f[keep], xs, offs, ref, w=w, kappa=kappa, phi=phi)
