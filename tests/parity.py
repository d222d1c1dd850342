"""Shared parity checks of GPU trajectories against the FP64 oracle.

Tolerances (per robot):
  positions: max_i |x_gpu - x_ref|_inf / (edge * max(nx, ny, nz)) < 1e-4
  fitness:   |f_gpu - f_ref| / max(|f_ref|, 1e-3 * edge) < 1e-3

The contact model switches between stick and slip discontinuously, so a robot whose trajectory
passes a switch within the float32 rounding of its state has no well-conditioned answer: the
oracle itself moves by more than the tolerance when its initial pose is perturbed by 1e-9 m
(below float32 resolution of the positions).  A robot that misses the tolerance is therefore
checked against the oracle's own conditioning: K oracle runs from initial poses perturbed by
1e-9 m; it is accepted if one of them meets the tolerance against the GPU result, or if the GPU
result is no farther from the unperturbed oracle than the perturbed oracle runs are from each
other (the spread the problem itself shows under an imperceptible input change).  Such robots
are counted, and their number is bounded by the caller.

Over thousands of steps the float32 rounding of every step is itself a perturbation of the
order of the positions' float32 resolution (1e-7 m at 1 m), far above 1e-9 m, so long runs
sample the envelope at that scale (`perturb`).  The spread is the largest pairwise distance
among K + 1 oracle runs, so one more independent run lands beyond it with probability about
2 / (K + 2); `envelope` scales it (1.5 by default, 2 for the long runs, where every robot is
checked this way).
"""
import numpy as np

POS_TOL = 1e-4
FIT_TOL = 1e-3
PERTURB = 1e-9


def pos_err(xg, xr, scale):
    if xr.size == 0:
        return 0.0
    return float(np.abs(xg.astype(np.float64) - xr).max()) / scale


def fit_err(f, fr, edge):
    if np.isinf(f) and np.isinf(fr) and np.sign(f) == np.sign(fr):
        return 0.0
    return abs(f - fr) / max(abs(fr), 1e-3 * edge)


def check_population(orc, pop, phys, nsteps, f_gpu, x_gpu, off, ref, w=None, kappa=None, phi=None,
                     K=8, max_sensitive_frac=0.1, perturb=PERTURB, envelope=1.5):
    """Assert parity for every robot; returns (index, errors, spreads) of the robots accepted
    through the envelope."""
    sensitive = []
    rng = np.random.default_rng(1234)
    for r in range(pop.P):
        scale = phys.edge * float(pop.dims[r].max())
        xg = x_gpu[off[r]:off[r + 1]]
        xr = ref["x"][r] if "x" in ref else None
        pe = pos_err(xg, xr, scale) if xr is not None else 0.0
        fe = fit_err(f_gpu[r], ref["fitness"][r], phys.edge)
        if pe < POS_TOL and fe < FIT_TOL:
            continue
        a, b = pop.voxel_off[r], pop.voxel_off[r + 1]
        kw = {}
        for name, arr in (("w", w), ("kappa", kappa), ("phi", phi)):
            if arr is not None:
                kw[name] = np.asarray(arr)[a:b]
        runs = []
        for _ in range(K):
            R = orc.Robot(pop.grid(r), pop.dims[r], phys, **kw)
            x0, v0 = R.state()
            R.set_state(x0 + rng.normal(0.0, perturb, x0.shape), v0, 0)
            R.simulate(nsteps)
            runs.append((R.state()[0], R.fitness()))
        near = min((pos_err(xg, xp, scale) if xr is not None else 0.0, fit_err(f_gpu[r], fp, phys.edge))
                   for xp, fp in runs)
        everyone = ([(xr, ref["fitness"][r])] if xr is not None else []) + runs
        spread_p = max((pos_err(p1.astype(np.float32), p2, scale) for p1, _ in everyone for p2, _ in everyone),
                       default=0.0) if xr is not None else 0.0
        spread_f = max(fit_err(f1, f2, phys.edge) for _, f1 in everyone for _, f2 in everyone)
        ok = (near[0] < POS_TOL and near[1] < FIT_TOL) or \
             (pe <= max(POS_TOL, envelope * spread_p) and fe <= max(FIT_TOL, envelope * spread_f))
        assert ok, (f"robot {r} dims {tuple(pop.dims[r])}: position error {pe:.3e}, fitness error "
                    f"{fe:.3e}; nearest perturbed oracle run {near[0]:.3e}, {near[1]:.3e}; oracle "
                    f"spread {spread_p:.3e}, {spread_f:.3e}")
        sensitive.append((r, round(pe, 6), round(fe, 6), round(float(spread_p), 6), round(float(spread_f), 6)))
    assert len(sensitive) <= max(1, int(max_sensitive_frac * pop.P)), \
        f"too many robots only within the perturbation envelope (robot, pos err, fit err, spreads): {sensitive}"
    return sensitive


def oracle_corner_modes(orc, grid, dims, nsteps, base, phys=None):
    """The contact modes of the oracle's FP64 run of one robot, laid out [nsteps][grid corners]
    (0 where no mass) as sim_impose_contact_modes takes them."""
    if phys is None:
        from paper_2405_00698_gb300 import workloads
        phys = workloads.CONFIG
    _, modes, _ = orc.fitness_after_modes(grid, dims, phys, nsteps, **base)
    mc = orc.Robot(grid, dims, phys, **base).topology()["mass_corner"]
    C = int(np.prod(np.asarray(dims) + 1))
    out = np.zeros((nsteps, C), np.uint8)
    out[:, mc] = modes
    return out


def robot_params(pop, r, w, kappa, phi):
    """Robot r's per-voxel (w, kappa, phi) as FP64 arrays for the oracle."""
    a, b = pop.voxel_off[r], pop.voxel_off[r + 1]
    return {"w": w[a:b].astype(np.float64), "kappa": kappa[a:b].astype(np.float64),
            "phi": phi[a:b].astype(np.float64)}
