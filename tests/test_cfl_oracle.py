"""Adaptive time step of Sec. 3.1.4 in the oracle: dt = min(dt_max, alpha dx / v_max)
against closed forms (particles at rest, a uniform velocity) and its step-to-step
consistency with the oracle's own particle velocities."""
import numpy as np
import pytest

import oracle as O
from paper_2404_01931_gb300 import scenes as S


def test_cfl_dt_closed_forms():
    n = 32
    sc = S.box(n, (0.3, 0.3, 0.3), (0.6, 0.6, 0.6), velocity=(0.0, -40.0, 0.0))
    p = O.Params(n=(n, n, n), dx=1.0 / n, cfl=3.0)
    r = O.step(p, *sc.arrays(), fields=False)
    assert r.dt == 3.0 * (1.0 / n) / 40.0          # alpha dx / |v|, below 1/240
    rest = S.box(n, (0.3, 0.3, 0.3), (0.6, 0.6, 0.6))
    assert O.step(p, *rest.arrays(), fields=False).dt == p.dt     # at rest: dt_max
    slow = S.box(n, (0.3, 0.3, 0.3), (0.6, 0.6, 0.6), velocity=(1.0, 0.0, 0.0))
    assert O.step(p, *slow.arrays(), fields=False).dt == p.dt     # limit above dt_max
    fixed = O.Params(n=(n, n, n), dx=1.0 / n)
    assert O.step(fixed, *sc.arrays(), fields=False).dt == fixed.dt


def test_cfl_dt_follows_the_particle_speeds():
    n = 24
    sc = S.random_velocities(S.dam_break(n), 35.0, seed=2)
    p = O.Params(n=(n, n, n), dx=1.0 / n, cfl=3.0)
    arrs = [a.astype(np.float64) for a in sc.arrays()]
    for _ in range(4):
        vmax = np.sqrt(arrs[3] ** 2 + arrs[4] ** 2 + arrs[5] ** 2).max()
        r = O.step(p, *arrs, fields=False)
        assert r.dt == pytest.approx(min(p.dt, 3.0 / n / vmax), rel=1e-15)
        assert r.dt < p.dt
        arrs = [r.x, r.y, r.z, r.u, r.v, r.w]


def test_cfl_step_equals_a_fixed_step_of_that_dt():
    """The adaptive step is the fixed step with its dt: same fields to rounding."""
    n = 16
    sc = S.random_velocities(S.box(n, (0.1, 0.0, 0.1), (0.7, 0.6, 0.8)), 30.0, seed=4)
    pa = O.Params(n=(n, n, n), dx=1.0 / n, cfl=2.0, cg_tol=1e-12)
    ra = O.step(pa, *sc.arrays())
    pf = O.Params(n=(n, n, n), dx=1.0 / n, dt=ra.dt, cg_tol=1e-12)
    rf = O.step(pf, *sc.arrays())
    assert np.abs(ra.pressure - rf.pressure).max() <= 1e-12 * np.abs(rf.pressure).max()
    assert np.abs(ra.y - rf.y).max() <= 1e-14
