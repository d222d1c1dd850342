"""ctypes wrapper of the FP64 CPU oracle (voxsim_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the test-suite, the smoke check and the CPU-baseline leg of
the benchmark, never by the library.  It shares no code with the CUDA path; parameters arrive as
plain attribute bags (any object with the Physics fields) and arrays as numpy buffers.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "voxsim_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liboracle.so")
GENOME_LEN = 20998

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FMA contraction, OpenMP over robots)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= os.path.getmtime(SRC):
        return LIB_PATH
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fopenmp", "-fPIC",
           "-shared", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class OrcParams(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("dt", "gravity", "mass", "edge", "damping", "k_ground",
                                           "mu_s", "mu_k", "freq", "dead_bound")] + [
        ("k_mat", C.c_double * 5), ("amp_mat", C.c_double * 5), ("phase_mat", C.c_double * 5),
        ("ground_on", C.c_int32), ("pad_", C.c_int32), ("spring_zeta", C.c_double),
        ("ground_zeta", C.c_double)]

    @classmethod
    def of(cls, phys) -> "OrcParams":
        p = cls()
        for n in ("dt", "gravity", "mass", "edge", "damping", "k_ground", "mu_s", "mu_k", "freq",
                  "dead_bound"):
            setattr(p, n, float(getattr(phys, n)))
        p.k_mat = (C.c_double * 5)(*[float(v) for v in phys.k_mat])
        p.amp_mat = (C.c_double * 5)(*[float(v) for v in phys.amp_mat])
        p.phase_mat = (C.c_double * 5)(*[float(v) for v in phys.phase_mat])
        p.ground_on = 1 if phys.ground_on else 0
        p.spring_zeta = float(getattr(phys, "spring_zeta", 0.0))
        p.ground_zeta = float(getattr(phys, "ground_zeta", 0.0))
        return p


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB_PATH)
            vp, i32, i64, u64, u32, d = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_uint32, C.c_double
            L.orc_round_bf16.argtypes = [d]; L.orc_round_bf16.restype = d
            L.orc_pe_table.argtypes = [i32, i32, i32, vp, vp]; L.orc_pe_table.restype = None
            L.orc_mlp_query.argtypes = [i32, i32, i32, vp, vp, vp, vp, vp, vp]; L.orc_mlp_query.restype = None
            L.orc_lcc_bfs.argtypes = [i32, i32, i32, vp, vp]; L.orc_lcc_bfs.restype = i32
            L.orc_lcc_unionfind.argtypes = [i32, i32, i32, vp, vp]; L.orc_lcc_unionfind.restype = i32
            L.orc_robot_new.argtypes = [i32, i32, i32, vp, vp, vp, vp, vp, i32]; L.orc_robot_new.restype = vp
            L.orc_robot_free.argtypes = [vp]; L.orc_robot_free.restype = None
            L.orc_robot_counts.argtypes = [vp, vp, vp]; L.orc_robot_counts.restype = None
            L.orc_robot_topology.argtypes = [vp] * 9; L.orc_robot_topology.restype = None
            L.orc_robot_get_state.argtypes = [vp, vp, vp]; L.orc_robot_get_state.restype = None
            L.orc_robot_set_state.argtypes = [vp, vp, vp, C.c_long]; L.orc_robot_set_state.restype = None
            L.orc_robot_simulate.argtypes = [vp, vp, i32]; L.orc_robot_simulate.restype = i32
            L.orc_robot_simulate_modes.argtypes = [vp, vp, i32, vp]; L.orc_robot_simulate_modes.restype = i32
            L.orc_robot_fitness.argtypes = [vp, vp]; L.orc_robot_fitness.restype = d
            L.orc_run_population.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp, i32, i32, i32, vp, vp, vp, vp, vp]
            L.orc_run_population.restype = i32
            L.orc_rng_draw.argtypes = [u64, u64, u64, u64, u64]; L.orc_rng_draw.restype = u32
            L.orc_evo_generation.argtypes = [i32, i32, vp, vp, vp, i32, u64, u64, u32, d, u32, vp, vp, vp, vp]
            L.orc_evo_generation.restype = i32
            L.orc_fitness_after.argtypes = [i32, i32, i32, vp, vp, vp, vp, vp, i32, i32, vp]
            L.orc_fitness_after.restype = d
            L.orc_fitness_after_modes.argtypes = [i32, i32, i32, vp, vp, vp, vp, vp, i32, i32, vp, vp, vp]
            L.orc_fitness_after_modes.restype = d
            L.orc_robot_adjoint.argtypes = [i32, i32, i32, vp, vp, vp, vp, vp, i32, i32, d, vp, vp, vp, vp]
            L.orc_robot_adjoint.restype = d
            L.orc_genome_diversity.argtypes = [i32, i32, vp]; L.orc_genome_diversity.restype = d
            L.orc_morphology_diversity.argtypes = [i32, i32, vp]; L.orc_morphology_diversity.restype = d
            _lib = L
    return _lib


def _f64(a, n=None):
    if a is None:
        return None
    out = np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(-1))
    if n is not None:
        assert out.size == n, (out.size, n)
    return out


def _grid(mat, dims):
    nx, ny, nz = (int(v) for v in dims)
    m = np.ascontiguousarray(np.asarray(mat, dtype=np.uint8).reshape(-1))
    assert m.size == nx * ny * nz
    return m, nx, ny, nz


# ------------------------------------------------------------------------------------------
# Encoding
# ------------------------------------------------------------------------------------------

def round_bf16(x: float) -> float:
    return lib().orc_round_bf16(float(x))


def pe_table(dims, B) -> np.ndarray:
    nx, ny, nz = (int(v) for v in dims)
    Bf = np.ascontiguousarray(np.asarray(B, dtype=np.float32))
    out = np.empty((nx * ny * nz, 256), dtype=np.float64)
    lib().orc_pe_table(nx, ny, nz, _p(Bf), _p(out))
    return out


def mlp_query(dims, B, genome):
    """Returns (materials u8 [Q], weight f64 [Q], outputs f64 [Q, 6], guard f64 [Q])."""
    nx, ny, nz = (int(v) for v in dims)
    Q = nx * ny * nz
    Bf = np.ascontiguousarray(np.asarray(B, dtype=np.float32))
    g = np.ascontiguousarray(np.asarray(genome, dtype=np.float32).reshape(-1))
    assert g.size == GENOME_LEN
    mat = np.empty(Q, np.uint8); w = np.empty(Q, np.float64)
    logits = np.empty((Q, 6), np.float64); guard = np.empty(Q, np.float64)
    lib().orc_mlp_query(nx, ny, nz, _p(Bf), _p(g), _p(mat), _p(w), _p(logits), _p(guard))
    return mat, w, logits, guard


# ------------------------------------------------------------------------------------------
# Components, robots
# ------------------------------------------------------------------------------------------

def lcc(mat, dims, method: str = "bfs") -> np.ndarray:
    m, nx, ny, nz = _grid(mat, dims)
    out = np.empty_like(m)
    fn = lib().orc_lcc_bfs if method == "bfs" else lib().orc_lcc_unionfind
    fn(nx, ny, nz, _p(m), _p(out))
    return out


class Robot:
    """One robot of the oracle.  w, kappa, phi: optional per-voxel float arrays."""

    def __init__(self, mat, dims, phys, w=None, kappa=None, phi=None, apply_lcc=True):
        self._m, nx, ny, nz = _grid(mat, dims)
        V = nx * ny * nz
        self._w, self._k, self._ph = _f64(w, V), _f64(kappa, V), _f64(phi, V)
        self._params = OrcParams.of(phys)
        self.dims = (nx, ny, nz)
        self._h = lib().orc_robot_new(nx, ny, nz, _p(self._m), _p(self._w), _p(self._k),
                                      _p(self._ph), C.byref(self._params), int(bool(apply_lcc)))
        M, S = C.c_int32(), C.c_int32()
        lib().orc_robot_counts(self._h, C.byref(M), C.byref(S))
        self.M, self.S = M.value, S.value

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_robot_free(h)
            self._h = None

    def topology(self):
        V = int(np.prod(self.dims))
        kept = np.empty(V, np.uint8); mc = np.empty(self.M, np.int32)
        sa = np.empty(self.S, np.int32); sb = np.empty(self.S, np.int32)
        L0, k, al, be = (np.empty(self.S, np.float64) for _ in range(4))
        lib().orc_robot_topology(self._h, _p(kept), _p(mc), _p(sa), _p(sb), _p(L0), _p(k), _p(al), _p(be))
        return dict(kept=kept, mass_corner=mc, a=sa, b=sb, L0=L0, k=k, alpha=al, beta=be)

    def state(self):
        x = np.empty((self.M, 3)); v = np.empty((self.M, 3))
        lib().orc_robot_get_state(self._h, _p(x), _p(v))
        return x, v

    def set_state(self, x, v, step: int):
        x = _f64(x, 3 * self.M); v = _f64(v, 3 * self.M)
        lib().orc_robot_set_state(self._h, _p(x), _p(v), int(step))

    def simulate(self, nsteps: int) -> int:
        return lib().orc_robot_simulate(self._h, C.byref(self._params), int(nsteps))

    def simulate_modes(self, force) -> int:
        """Step once per row of force (uint8 [nsteps, M], mass order) with those contact modes
        imposed."""
        fm = np.ascontiguousarray(np.asarray(force, dtype=np.uint8).reshape(-1, self.M))
        return lib().orc_robot_simulate_modes(self._h, C.byref(self._params), int(fm.shape[0]), _p(fm))

    def fitness(self) -> float:
        return lib().orc_robot_fitness(self._h, C.byref(self._params))


def run_population(pop, phys, nsteps: int, w=None, kappa=None, phi=None, apply_lcc=True,
                   nthreads: int = 0, want_x: bool = False):
    """Simulate every robot of a workloads.Population.  Returns dict(fitness, M, S, threads,
    x (list of [M_r, 3] arrays if want_x))."""
    P = pop.P
    dims = np.ascontiguousarray(pop.dims, dtype=np.int32)
    voff = np.ascontiguousarray(pop.voxel_off, dtype=np.int64)
    mats = np.ascontiguousarray(pop.mats, dtype=np.uint8)
    n = mats.size
    w, kappa, phi = _f64(w, n), _f64(kappa, n), _f64(phi, n)
    fit = np.empty(P); M = np.empty(P, np.int32); S = np.empty(P, np.int32)
    params = OrcParams.of(phys)
    moff = xout = None
    if want_x:
        caps = [(int(a) + 1) * (int(b) + 1) * (int(c) + 1) for a, b, c in pop.dims]
        moff = np.zeros(P + 1, np.int64); moff[1:] = np.cumsum(caps)
        xout = np.zeros((int(moff[-1]), 3))
    used = lib().orc_run_population(P, _p(dims), _p(voff), _p(mats), _p(w), _p(kappa), _p(phi),
                                    C.byref(params), int(bool(apply_lcc)), int(nsteps), int(nthreads),
                                    _p(fit), _p(M), _p(S), _p(moff), _p(xout))
    out = dict(fitness=fit, M=M, S=S, threads=used)
    if want_x:
        out["x"] = [xout[moff[r]:moff[r] + M[r]] for r in range(P)]
    return out


# ------------------------------------------------------------------------------------------
# Evolution
# ------------------------------------------------------------------------------------------

def rng_draw(seed: int, gen: int, child: int, gene: int, purpose: int) -> int:
    return int(lib().orc_rng_draw(seed, gen, child, gene, purpose))


def evo_generation(fitness, genomes, E: int, seed: int, gen: int, mut_threshold: int, sigma: float,
                   keep_threshold: int = 0):
    """Returns dict(genomes f64 [P, G], order i32 [P], parents i32 [P, 2], mask u8 [P, G],
    mutate u8 [P, G])."""
    f = _f64(fitness)
    g = np.ascontiguousarray(np.asarray(genomes, dtype=np.float32))
    P, G = g.shape
    out = np.empty((P, G)); order = np.empty(P, np.int32); par = np.empty((P, 2), np.int32)
    mask = np.empty((P, G), np.uint8); mut = np.empty((P, G), np.uint8)
    rc = lib().orc_evo_generation(P, G, _p(f), _p(g), _p(out), int(E), int(seed), int(gen),
                                  int(mut_threshold), float(sigma), int(keep_threshold), _p(order),
                                  _p(par), _p(mask), _p(mut))
    if rc != 0:
        raise ValueError("bad evolution sizes")
    return dict(genomes=out, order=order, parents=par, mask=mask, mutate=mut)


# ------------------------------------------------------------------------------------------
# Differentiation
# ------------------------------------------------------------------------------------------

def fitness_after(mat, dims, phys, nsteps, w=None, kappa=None, phi=None, apply_lcc=True):
    """(fitness, contact-mode hash) of a fresh robot after nsteps."""
    m, nx, ny, nz = _grid(mat, dims)
    V = m.size
    w, kappa, phi = _f64(w, V), _f64(kappa, V), _f64(phi, V)
    h = C.c_uint64()
    params = OrcParams.of(phys)
    f = lib().orc_fitness_after(nx, ny, nz, _p(m), _p(w), _p(kappa), _p(phi), C.byref(params),
                                int(bool(apply_lcc)), int(nsteps), C.byref(h))
    return f, h.value


def fitness_after_modes(mat, dims, phys, nsteps, w=None, kappa=None, phi=None, apply_lcc=True,
                        force=None):
    """(fitness, modes uint8 [nsteps, M] in mass order, contact-mode hash) of a fresh robot after
    nsteps; with `force` ([nsteps, M] uint8) the contact modes are imposed instead of decided."""
    m, nx, ny, nz = _grid(mat, dims)
    V = m.size
    w, kappa, phi = _f64(w, V), _f64(kappa, V), _f64(phi, V)
    R = Robot(mat, dims, phys, w=w, kappa=kappa, phi=phi, apply_lcc=apply_lcc)
    M = R.M
    del R
    out = np.zeros((max(nsteps, 1), max(M, 1)), np.uint8)
    fm = None
    if force is not None:
        fm = np.ascontiguousarray(np.asarray(force, dtype=np.uint8).reshape(nsteps, M))
    h = C.c_uint64()
    params = OrcParams.of(phys)
    f = lib().orc_fitness_after_modes(nx, ny, nz, _p(m), _p(w), _p(kappa), _p(phi), C.byref(params),
                                      int(bool(apply_lcc)), int(nsteps), _p(fm), _p(out), C.byref(h))
    return f, out[:nsteps, :M], h.value


def adjoint(mat, dims, phys, nsteps, dL_df=1.0, w=None, kappa=None, phi=None, apply_lcc=True,
            lx_final=None):
    """(fitness, g_w, g_kappa, g_phi) per voxel of L = dL_df * fitness, or of
    L = sum lx_final . x(N) when lx_final ([M, 3]) is given."""
    m, nx, ny, nz = _grid(mat, dims)
    V = m.size
    w, kappa, phi = _f64(w, V), _f64(kappa, V), _f64(phi, V)
    lxf = _f64(lx_final)
    gw, gk, gp = np.empty(V), np.empty(V), np.empty(V)
    params = OrcParams.of(phys)
    f = lib().orc_robot_adjoint(nx, ny, nz, _p(m), _p(w), _p(kappa), _p(phi), C.byref(params),
                                int(bool(apply_lcc)), int(nsteps), float(dL_df), _p(lxf),
                                _p(gw), _p(gk), _p(gp))
    return f, gw, gk, gp


# ------------------------------------------------------------------------------------------
# Diversity
# ------------------------------------------------------------------------------------------

def genome_diversity(genomes) -> float:
    g = np.ascontiguousarray(np.asarray(genomes, dtype=np.float32))
    return lib().orc_genome_diversity(g.shape[0], g.shape[1], _p(g))


def morphology_diversity(mats) -> float:
    """mats: uint8 [P, V] material grids of one shape."""
    m = np.ascontiguousarray(np.asarray(mats, dtype=np.uint8))
    return lib().orc_morphology_diversity(m.shape[0], m.shape[1], _p(m))
