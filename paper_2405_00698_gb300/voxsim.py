"""Python binding of libvoxsim.so (include/voxsim.h).  Argument marshalling only: every step of
the path runs in the library's CUDA kernels.  PyTorch supplies device memory and streams.

The binding fails loudly when the compiled library is missing; there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libvoxsim.so")

SIM_OK, SIM_EINVAL, SIM_ENOMEM, SIM_ECUDA, SIM_ESTATE, SIM_ETIMEOUT, SIM_ENUMERIC = range(7)
MEM_HOST, MEM_DEVICE = 0, 1
MODE_MATERIALS, MODE_LOGITS, MODE_MLP, MODE_PARAMS, MODE_PARAM_ROWS = 0, 1, 2, 3, 4
ACC_AUTO, ACC_ATOMIC, ACC_GATHER = 0, 1, 2
MLP_TENSOR, MLP_SIMT = 0, 1
PATH_AUTO, PATH_RESIDENT, PATH_STREAMED, PATH_PLAIN = 0, 1, 2, 3
LATTICE_AUTO, LATTICE_CORNER, LATTICE_COMPACT, LATTICE_PACKED = 0, 1, 2, 3
GENOME_LEN = 20998

EXPORTS = ("sim_create", "sim_destroy", "sim_last_error", "sim_set_population", "sim_step_n",
           "sim_fitness", "evo_generation", "evo_generation_static", "evo_gradient_step", "sim_set_checkpointing",
           "sim_set_trajectory_records", "sim_backward", "sim_get_contact_modes", "sim_autotune", "sim_diversity", "sim_get_counts", "sim_get_state", "sim_get_voxels", "sim_get_topology",
           "sim_get_timing", "sim_check_status_words", "sim_impose_contact_modes", "evo_elite_weights",
           "sim_measure_smem_bandwidth")


class VoxsimError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"voxsim status {status}: {msg}")
        self.status = status


class SimParams(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("dt", "gravity", "mass", "edge", "damping", "k_ground",
                                           "mu_s", "mu_k", "freq", "dead_bound")] + [
        ("k_mat", C.c_double * 5), ("amp_mat", C.c_double * 5), ("phase_mat", C.c_double * 5),
        ("ground_on", C.c_int32), ("accumulate", C.c_int32), ("path", C.c_int32),
        ("threads", C.c_int32), ("mlp_kernel", C.c_int32), ("lattice", C.c_int32),
        ("spring_zeta", C.c_double), ("ground_zeta", C.c_double)]

    @classmethod
    def of(cls, phys, accumulate: int = ACC_AUTO, path: int = PATH_AUTO, threads: int = 0,
           mlp_kernel: int = 0, lattice: int = 0):
        p = cls()
        for n in ("dt", "gravity", "mass", "edge", "damping", "k_ground", "mu_s", "mu_k", "freq",
                  "dead_bound"):
            setattr(p, n, float(getattr(phys, n)))
        p.k_mat = (C.c_double * 5)(*map(float, phys.k_mat))
        p.amp_mat = (C.c_double * 5)(*map(float, phys.amp_mat))
        p.phase_mat = (C.c_double * 5)(*map(float, phys.phase_mat))
        p.ground_on = 1 if phys.ground_on else 0
        p.accumulate, p.path, p.threads = int(accumulate), int(path), int(threads)
        p.mlp_kernel = int(mlp_kernel)
        p.lattice = int(lattice)
        p.spring_zeta = float(getattr(phys, "spring_zeta", 0.0))
        p.ground_zeta = float(getattr(phys, "ground_zeta", 0.0))
        return p


class VoxelParams(C.Structure):
    _fields_ = [("mat", C.c_void_p), ("w", C.c_void_p), ("kappa", C.c_void_p), ("phi", C.c_void_p)]


class ParamRows(C.Structure):
    _fields_ = [("mat", C.c_void_p), ("rows", C.c_void_p)]


class EvoParams(C.Structure):
    _fields_ = [("elites", C.c_int32), ("mut_threshold", C.c_uint32), ("sigma", C.c_float),
                ("keep_threshold", C.c_uint32), ("seed", C.c_uint64)]


_lib = None


def lib():
    """Load libvoxsim.so (built in-tree by paper_2405_00698_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built: run paper_2405_00698_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        vp, i32, u64 = C.c_void_p, C.c_int32, C.c_uint64
        sig = {
            "sim_create": [vp, i32, vp, vp],
            "sim_destroy": [vp],
            "sim_set_population": [vp, i32, vp, i32, vp, vp, i32],
            "sim_step_n": [vp, i32],
            "sim_fitness": [vp, vp, i32],
            "evo_generation": [vp, vp, vp, vp, i32, i32, vp, u64, vp, vp],
            "evo_generation_static": [vp, vp, vp, i32, i32, vp, u64, vp, vp, vp],
            "evo_gradient_step": [vp, vp, i32, i32, vp, vp, vp, vp, i32, C.c_float, C.c_float, C.c_float,
                                  vp, vp],
            "sim_set_checkpointing": [vp, i32],
            "sim_set_trajectory_records": [vp, i32],
            "sim_backward": [vp, vp, vp, vp, vp],
            "sim_get_contact_modes": [vp, i32, vp],
            "sim_autotune": [vp, i32, vp, vp],
            "sim_diversity": [vp, vp, i32, i32, vp],
            "sim_get_counts": [vp, vp, vp],
            "sim_get_state": [vp, vp, vp, vp, i32],
            "sim_get_voxels": [vp, vp, vp, vp, vp, vp],
            "sim_get_topology": [vp, vp, vp, vp],
            "sim_get_timing": [vp, vp, vp],
            "sim_check_status_words": [vp],
            "sim_impose_contact_modes": [vp, i32, vp, i32],
            "evo_elite_weights": [vp, vp, i32, i32, vp],
            "sim_measure_smem_bandwidth": [vp, vp],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = C.c_int32
        L.sim_last_error.argtypes = [vp]
        L.sim_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def _check(status: int):
    if status != SIM_OK:
        raise VoxsimError(status, lib().sim_last_error(None).decode())


def _ptr(a):
    """(pointer, mem) of a torch tensor (device or CPU) or numpy array; None -> (None, host)."""
    if a is None:
        return None, MEM_HOST
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"], "numpy input must be C-contiguous"
        return a.ctypes.data, MEM_HOST
    import torch
    if isinstance(a, torch.Tensor):
        assert a.is_contiguous(), "tensor input must be contiguous"
        return a.data_ptr(), (MEM_DEVICE if a.is_cuda else MEM_HOST)
    raise TypeError(type(a))


class Simulator:
    """One library context on one GPU, enqueueing on a torch CUDA stream."""

    def __init__(self, phys, device: int = 0, stream=None, accumulate: int = ACC_AUTO,
                 path: int = PATH_AUTO, threads: int = 0, mlp_kernel: int = MLP_TENSOR,
                 lattice: int = 0):
        import torch
        self.device = int(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.params = SimParams.of(phys, accumulate, path, threads, mlp_kernel, lattice)
        h = C.c_void_p()
        _check(lib().sim_create(C.byref(self.params), self.device, C.c_void_p(self.stream.cuda_stream),
                                C.byref(h)))
        self._h = h
        self.P = 0
        self.dims = None
        self.voxel_off = None

    def close(self):
        if getattr(self, "_h", None):
            lib().sim_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- population ------------------------------------------------------------------------
    def set_population(self, dims, genomes, mode: int = MODE_MATERIALS, B=None):
        """dims: [P, 3] ints.  genomes: per mode (numpy host array or torch tensor)."""
        d = np.ascontiguousarray(np.asarray(dims, dtype=np.int32).reshape(-1, 3))
        P = d.shape[0]
        keep = [d]
        if mode == MODE_PARAM_ROWS:
            mat, rows = genomes
            ptrs = [_ptr(mat), _ptr(rows)]
            mems = {m for _, m in ptrs}
            assert len(mems) == 1, "materials and rows must both be host or both device"
            pr = ParamRows(*[p for p, _ in ptrs])
            keep += [pr, mat, rows]
            gptr, mem = C.addressof(pr), mems.pop()
        elif mode == MODE_PARAMS:
            mat, w, kappa, phi = genomes
            ptrs = [_ptr(mat), _ptr(w), _ptr(kappa), _ptr(phi)]
            mems = {m for _, m in ptrs}
            assert len(mems) == 1, "per-voxel arrays must all be host or all device"
            vp = VoxelParams(*[p for p, _ in ptrs])
            keep += [vp, mat, w, kappa, phi]
            gptr, mem = C.addressof(vp), mems.pop()
        else:
            gptr, mem = _ptr(genomes)
            keep.append(genomes)
        bptr = None
        if B is not None:
            bptr, bmem = _ptr(B)
            assert bmem == mem, "B must be in the same memory as the genomes"
            keep.append(B)
        self._sync_inputs(mem)
        _check(lib().sim_set_population(self._h, P, d.ctypes.data, int(mode), gptr, bptr, mem))
        self.P = P
        self.dims = d
        sizes = d.prod(axis=1).astype(np.int64)
        self.voxel_off = np.concatenate([[0], np.cumsum(sizes)])
        self._keep = keep   # host buffers stay alive until the next population

    def set_population_from(self, pop, mode: int = MODE_MATERIALS, genomes=None, B=None):
        """From a workloads.Population (materials, or another mode's genomes)."""
        return self.set_population(pop.dims, pop.mats if genomes is None else genomes, mode, B)

    def _sync_inputs(self, mem):
        if mem == MEM_DEVICE:
            import torch
            # inputs written on torch's current stream must be ready on the library's stream
            cur = torch.cuda.current_stream(self.device)
            if cur != self.stream:
                self.stream.wait_stream(cur)

    # -- stepping ----------------------------------------------------------------------------
    def step(self, n: int):
        _check(lib().sim_step_n(self._h, int(n)))

    def fitness(self, out=None):
        """FP64 fitness per robot; into `out` (CUDA tensor) or returned as numpy."""
        if out is None:
            res = np.empty(self.P, np.float64)
            _check(lib().sim_fitness(self._h, res.ctypes.data, MEM_HOST))
            return res
        p, mem = _ptr(out)
        _check(lib().sim_fitness(self._h, p, mem))
        return out

    def autotune(self, n_steps: int = 50):
        """Time the admissible stepping kernels per size class and keep the fastest; returns
        (kind [10], threads [10]) with kind 0 lattice per corner, 1 atomic resident, 2 streamed,
        3 lattice direction-compacted, 4 cluster of lattice blocks, 5 lattice in mass-sized
        thread groups (sparse robots of more than 768 corners)."""
        kind = np.zeros(10, np.int32); threads = np.zeros(10, np.int32)
        _check(lib().sim_autotune(self._h, int(n_steps), kind.ctypes.data, threads.ctypes.data))
        return kind, threads

    def diversity(self, genomes=None, P: Optional[int] = None):
        """(genome RMS pairwise distance, morphology mean pairwise disagreement fraction)."""
        out = np.empty(2, np.float64)
        if genomes is not None:
            P_, G = genomes.shape
            ptr = _ptr(genomes)[0]
        else:
            P_, G, ptr = (P if P is not None else self.P), 0, None
        _check(lib().sim_diversity(self._h, ptr, int(P_), int(G), out.ctypes.data))
        return float(out[0]), float(out[1])

    def counts(self):
        M = np.empty(self.P, np.int32); S = np.empty(self.P, np.int32)
        _check(lib().sim_get_counts(self._h, M.ctypes.data, S.ctypes.data))
        return M, S

    def state(self):
        """(x [sum M, 3], v [sum M, 3], offsets [P+1]) on the host."""
        M, _ = self.counts()
        tot = int(M.sum())
        x = np.empty((tot, 3), np.float32); v = np.empty((tot, 3), np.float32)
        off = np.empty(self.P + 1, np.int32)
        _check(lib().sim_get_state(self._h, x.ctypes.data, v.ctypes.data, off.ctypes.data, MEM_HOST))
        return x, v, off

    def voxels(self):
        n = int(self.voxel_off[-1])
        dec = np.empty(n, np.uint8); kept = np.empty(n, np.uint8)
        w = np.empty(n, np.float32); k = np.empty(n, np.float32); ph = np.empty(n, np.float32)
        _check(lib().sim_get_voxels(self._h, dec.ctypes.data, kept.ctypes.data, w.ctypes.data,
                                    k.ctypes.data, ph.ctypes.data))
        return dict(decoded=dec, kept=kept, w=w, kappa=k, phi=ph)

    def topology(self):
        M, S = self.counts()
        mc = np.empty(int(M.sum()), np.int32)
        ab = np.empty((int(S.sum()), 2), np.int32)
        sp = np.empty((int(S.sum()), 4), np.float32)
        _check(lib().sim_get_topology(self._h, mc.ctypes.data, ab.ctypes.data, sp.ctypes.data))
        return dict(M=M, S=S, mass_corner=mc, ab=ab, params=sp)

    def measure_smem_bandwidth(self) -> float:
        """Measured shared-memory bandwidth of the device, GB/s over all SMs."""
        g = C.c_double()
        _check(lib().sim_measure_smem_bandwidth(self._h, C.byref(g)))
        return g.value

    def timing(self):
        ms = C.c_double(); n = C.c_int64()
        _check(lib().sim_get_timing(self._h, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    # -- differentiation ---------------------------------------------------------------------
    def set_checkpointing(self, k: int):
        _check(lib().sim_set_checkpointing(self._h, int(k)))

    def set_trajectory_records(self, on: bool):
        """Keep every step's record of the recorded run, so that backward needs no replay."""
        _check(lib().sim_set_trajectory_records(self._h, 1 if on else 0))

    def impose_contact_modes(self, robot: int, modes):
        """Impose contact modes on one robot's first steps (uint8 [n_steps, corners] in the
        layout of contact_modes); None clears every imposition."""
        if modes is None:
            _check(lib().sim_impose_contact_modes(self._h, 0, None, 0))
            return
        m = np.ascontiguousarray(modes, dtype=np.uint8)
        _check(lib().sim_impose_contact_modes(self._h, int(robot), m.ctypes.data, int(m.shape[0])))

    def contact_modes(self, robot: int, n_steps: int):
        """Contact mode (0 free, 1 stuck, 2 slipping, 3 slipping with the kinetic friction
        saturated) of every grid corner of one robot at every
        step of the recorded run: uint8 [n_steps, corners]."""
        nx, ny, nz = (int(v) for v in self.dims[robot])
        out = np.zeros((n_steps, (nx + 1) * (ny + 1) * (nz + 1)), np.uint8)
        _check(lib().sim_get_contact_modes(self._h, int(robot), out.ctypes.data))
        return out

    def backward(self, dL_df, g_w, g_kappa, g_phi):
        ptrs = [_ptr(t)[0] for t in (dL_df, g_w, g_kappa, g_phi)]
        _check(lib().sim_backward(self._h, *ptrs))

    # -- evolution ---------------------------------------------------------------------------
    def evo_generation(self, fitness, genomes_in, genomes_out, evo, generation: int,
                       parents=None, mask=None):
        """All tensors on the device: fitness f64 [P], genomes f32 [P, G] (in and out may be the
        same tensor; genomes_in None: the genome rows the last set_population read from host
        memory), parents i32 [P, 2] or None, mask u8 [P, G] or None."""
        P, G = genomes_out.shape
        e = EvoParams(int(evo.elites(P)), int(evo.mut_threshold()), float(evo.sigma),
                      int(evo.keep_threshold()), int(evo.seed))
        self._sync_inputs(MEM_DEVICE)
        _check(lib().evo_generation(self._h, _ptr(fitness)[0], _ptr(genomes_in)[0],
                                    _ptr(genomes_out)[0], int(P), int(G), C.byref(e),
                                    int(generation), _ptr(parents)[0], _ptr(mask)[0]))


    def evo_elite_weights(self, fitness, E: int, out):
        """out[r] = 1 for the E best robots with finite fitness (evo_generation's rank order), else
        0 (device f64 tensors [P]); the adjoint weights of the elites' summed fitness."""
        P = fitness.shape[0]
        self._sync_inputs(MEM_DEVICE)
        _check(lib().evo_elite_weights(self._h, _ptr(fitness)[0], int(P), int(E), _ptr(out)[0]))
        return out

    def evo_gradient_step(self, genomes, g_w, g_kappa, g_phi, eta, rows=None, lo=None, hi=None):
        """Lamarckian step on MODE_PARAM_ROWS genome rows (device f32 [P, 3V]) along sim_backward's
        per-voxel gradients: genome <- clamp(eta_seg * grad + genome, lo, hi) for the listed robots
        (host int sequence, None = all); eta = (eta_w, eta_kappa, eta_phi); lo / hi device f32
        [3V] or None."""
        ew, ek, ep = (float(e) for e in eta)
        P, G = genomes.shape
        rl = None if rows is None else np.ascontiguousarray(np.asarray(rows, dtype=np.int32))
        self._sync_inputs(MEM_DEVICE)
        _check(lib().evo_gradient_step(self._h, _ptr(genomes)[0], int(P), int(G), _ptr(g_w)[0],
                                       _ptr(g_kappa)[0], _ptr(g_phi)[0],
                                       None if rl is None else rl.ctypes.data,
                                       0 if rl is None else int(rl.size), ew, ek, ep,
                                       _ptr(lo)[0], _ptr(hi)[0]))


def fitness_function():
    """torch.autograd.Function: fitness of a population under the per-voxel parametrisation
    (materials, w, kappa, phi) after n steps, differentiable in (w, kappa, phi) through the
    library's checkpointed adjoint.

        f = fitness_function().apply(sim, dims, mats, w, kappa, phi, n_steps, k_ckpt)

    mats (uint8) and w, kappa, phi (float32) are CUDA tensors over all voxels; f is float64 [P]."""
    import torch

    class _Fitness(torch.autograd.Function):
        @staticmethod
        def forward(ctx, sim, dims, mats, w, kappa, phi, n_steps, k_ckpt):
            sim.set_checkpointing(int(k_ckpt))
            sim.set_population(dims, (mats, w.detach().contiguous(), kappa.detach().contiguous(),
                                      phi.detach().contiguous()), MODE_PARAMS)
            sim.step(int(n_steps))
            out = torch.empty(sim.P, dtype=torch.float64, device=w.device)
            sim.fitness(out)
            ctx.sim = sim
            ctx.nvox = w.numel()
            return out

        @staticmethod
        def backward(ctx, grad):
            sim = ctx.sim
            dev = grad.device
            gw = torch.empty(ctx.nvox, dtype=torch.float32, device=dev)
            gk = torch.empty_like(gw)
            gp = torch.empty_like(gw)
            sim.backward(grad.detach().to(torch.float64).contiguous(), gw, gk, gp)
            return None, None, None, gw, gk, gp, None, None

    return _Fitness
