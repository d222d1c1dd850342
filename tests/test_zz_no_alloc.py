"""The allocation-free evolution step (evo_generation_static), called through the C ABI, gives the
same generation as the context-based evo_generation, on two calls in a row.

It exists for callers that cannot allocate device memory: a process whose memory pool already
holds the whole device, where another cudaMalloc would fail, or a loop that must not allocate
once running, because cudaMalloc and cudaFree can synchronise the device.  Its only scratch is a
fixed array built into the library.  The two entry points run the same kernels on the same
inputs, so their results must agree bit for bit.  This file is named to be collected
last, so a failure here comes after every other test has run; it also passes on its own in a
fresh process."""
import ctypes as C

import numpy as np
import pytest

from paper_2405_00698_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_00698_gb300 import build, voxsim
    build.build()
    return voxsim


def test_static_scratch_generation_matches_context_generation(vs):
    import torch
    lib = vs.lib()
    rng = np.random.default_rng(90)
    P, G = 1024, W.GENOME_LEN
    evo = W.Evolution(seed=31)
    e = vs.EvoParams(evo.elites(P), evo.mut_threshold(), evo.sigma, 0, evo.seed)
    stream = torch.cuda.current_stream()
    sim = vs.Simulator(W.CONFIG, stream=stream)
    genomes = torch.from_numpy(W.mlp_genomes(rng, P)).cuda()
    for call in range(2):                      # two calls in a row share the static scratch
        fit = torch.from_numpy(np.round(rng.standard_normal(P), 2)).cuda()   # ties included
        ref = torch.empty_like(genomes)
        ref_par = torch.empty((P, 2), dtype=torch.int32, device="cuda")
        ref_mask = torch.empty((P, G), dtype=torch.uint8, device="cuda")
        sim.evo_generation(fit, genomes, ref, evo, call, ref_par, ref_mask)
        out = torch.empty_like(genomes)
        par = torch.empty_like(ref_par)
        mask = torch.empty_like(ref_mask)
        st = lib.evo_generation_static(fit.data_ptr(), genomes.data_ptr(), out.data_ptr(), P, G,
                                       C.byref(e), call, par.data_ptr(), mask.data_ptr(),
                                       C.c_void_p(stream.cuda_stream))
        assert st == vs.SIM_OK, lib.sim_last_error(None).decode()
        torch.cuda.synchronize()
        assert torch.equal(par, ref_par) and torch.equal(mask, ref_mask)
        assert torch.equal(out, ref)
        genomes = out
    # sizes beyond the built-in scratch are refused, not written past it
    big = torch.zeros(16385, dtype=torch.float64, device="cuda")
    g = torch.zeros((16385, 4), device="cuda")
    g2 = torch.empty_like(g)
    st = lib.evo_generation_static(big.data_ptr(), g.data_ptr(), g2.data_ptr(), 16385, 4, C.byref(e), 0,
                                   None, None, C.c_void_p(stream.cuda_stream))
    assert st == vs.SIM_EINVAL and b"16384" in lib.sim_last_error(None)
    sim.close()
