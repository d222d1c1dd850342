"""Shared parity checks of GPU trajectories against the FP64 oracle.

Tolerances (per robot):
  positions: max_i |x_gpu - x_ref|_inf / (edge * max(nx, ny, nz)) < 1e-4
  fitness:   |f_gpu - f_ref| / max(|f_ref|, 1e-3 * edge) < 1e-3

The contact model switches between stick and slip discontinuously, so a robot whose trajectory
passes a switch within the float32 rounding of its state has no well-conditioned answer: the
oracle itself moves by more than the tolerance when its initial pose is perturbed by 1e-9 m
(below float32 resolution of the positions).  A robot that misses the tolerance is therefore
accepted only if one of the oracle's own perturbed runs (K runs, initial pose perturbed by
1e-9 m) meets the tolerance against the GPU result; such robots are counted and reported, and
their number is bounded by the caller.
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
                     K=6, max_sensitive_frac=0.1):
    """Assert parity for every robot; returns the indices accepted through the envelope."""
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
        ok = False
        best = (pe, fe)
        for _ in range(K):
            R = orc.Robot(pop.grid(r), pop.dims[r], phys, **kw)
            x0, v0 = R.state()
            R.set_state(x0 + rng.normal(0.0, PERTURB, x0.shape), v0, 0)
            R.simulate(nsteps)
            xp, _ = R.state()
            pe2 = pos_err(xg, xp, scale) if xr is not None else 0.0
            fe2 = fit_err(f_gpu[r], R.fitness(), phys.edge)
            best = (min(best[0], pe2), min(best[1], fe2))
            if pe2 < POS_TOL and fe2 < FIT_TOL:
                ok = True
                break
        assert ok, (f"robot {r} dims {tuple(pop.dims[r])}: position error {pe:.3e}, fitness error "
                    f"{fe:.3e} (best within the oracle's perturbation envelope {best[0]:.3e}, {best[1]:.3e})")
        sensitive.append(r)
    assert len(sensitive) <= max(1, int(max_sensitive_frac * pop.P)), \
        f"too many robots only within the perturbation envelope: {sensitive}"
    return sensitive
