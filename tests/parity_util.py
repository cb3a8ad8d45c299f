"""Helpers shared by the GPU parity tests: run the CUDA path and the oracle on the
same seeded inputs and compare field by field."""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_2404_01931_gb300 import flip as F


def rel_l2(a, b, floor: float = 0.0) -> float:
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), floor, 1e-300))


def oracle_params(n, dx=None, **kw) -> O.Params:
    n = (n, n, n) if np.isscalar(n) else tuple(n)
    return O.Params(n=n, dx=1.0 / max(n) if dx is None else dx, **kw)


def flip_params(n, dx=None, **kw) -> F.FlipParams:
    n = (n, n, n) if np.isscalar(n) else tuple(n)
    p = F.default_params(*n)
    p.dx = 1.0 / max(n) if dx is None else dx
    p.skin = 1e-3 * p.dx
    for k, v in kw.items():
        if k == "gravity":
            for i in range(3):
                p.gravity[i] = v[i]
        else:
            setattr(p, k, v)
    return p


def matched(n, **kw):
    """(oracle params, library params) describing the same scene settings."""
    okw = {k: v for k, v in kw.items() if k in ("dt", "gravity", "rho", "flip_ratio", "cg_tol",
                                                "cg_max_iter", "advect_source", "skin",
                                                "preconditioner")}
    fkw = {k: v for k, v in kw.items() if k not in ("skin",)}
    fp = flip_params(n, **fkw)
    if "skin" in kw:
        fp.skin = kw["skin"]
    op = oracle_params(n, **okw)
    if "cg_max_iter" not in kw:
        op.cg_max_iter = fp.cg_max_iter
    op.preconditioner = fp.preconditioner
    op.mg_nu = fp.mg_smooth
    return op, fp


def gpu_step(fp, arrays, nsteps=1, fields=True, precision=None):
    """Runs nsteps on the GPU; returns a dict of fields (particles in creation order)."""
    if precision is not None:
        fp.precision = precision
    out = {}
    with F.Simulation(fp, *arrays) as sim:
        rc, st = sim.step(nsteps, stats=True)
        out["rc"], out["stats"] = rc, st
        out["particles"] = sim.particles()
        if fields:
            for name, f in (("u_old", (F.U_OLD, F.V_OLD, F.W_OLD)),
                            ("u_new", (F.U_NEW, F.V_NEW, F.W_NEW))):
                out[name] = [sim.read(x) for x in f]
            out["p"] = sim.read(F.PRESSURE_F64)
            out["rhs"] = sim.read(F.RHS)
            out["type"] = sim.read(F.CELL_TYPE)
    return out


def face_floor(n, dt=1 / 240, g=9.81):
    nf = (n[0] + 1) * n[1] * n[2] if not np.isscalar(n) else (n + 1) * n * n
    return g * dt * np.sqrt(nf)
