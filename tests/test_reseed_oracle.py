"""Reseeding (Sec. 3.1.2) in the oracle: cells below the minimum are refilled, cells
above the maximum are trimmed, and the new particles sit where the documented
SplitMix64 counter puts them, with the projected grid velocity."""
import numpy as np
import pytest

import oracle as O
from paper_2404_01931_gb300 import scenes as S


def _cells(p, x, y, z):
    n = p.n
    i = np.clip(np.floor(np.asarray(x, np.float64) * n[0]).astype(int), 0, n[0] - 1)
    j = np.clip(np.floor(np.asarray(y, np.float64) * n[1]).astype(int), 0, n[1] - 1)
    k = np.clip(np.floor(np.asarray(z, np.float64) * n[2]).astype(int), 0, n[2] - 1)
    return i + n[0] * (j + n[1] * k)


def test_lone_particles_at_rest_are_refilled_in_place():
    n = 16
    sc = S.box(n, (0.2, 0.0, 0.2), (0.7, 0.5, 0.8), density=1)        # one per cell
    p = O.Params(n=(n, n, n), dx=1 / n, gravity=(0.0, 0.0, 0.0), ppc_min=3, reseed_seed=9)
    r = O.step(p, *sc.arrays(), fields=False, step_index=5)
    assert r.status == 0
    nf = sc.fluid_mask.sum()
    assert r.added == 2 * nf and len(r.x) == 3 * nf
    counts = np.bincount(_cells(p, r.x, r.y, r.z), minlength=n ** 3)
    assert set(np.unique(counts)) == {0, 3}
    new = slice(sc.n_particles, None)
    assert np.all(r.u[new] == 0) and np.all(r.v[new] == 0) and np.all(r.w[new] == 0)


def test_new_particle_positions_follow_the_counter():
    n = 8
    sc = S.box(n, (0.25, 0.25, 0.25), (0.5, 0.5, 0.5), density=1)
    p = O.Params(n=(n, n, n), dx=1 / n, gravity=(0.0, 0.0, 0.0), ppc_min=2, reseed_seed=1234)
    step = 3
    r = O.step(p, *sc.arrays(), fields=False, step_index=step)
    cells = np.flatnonzero(sc.fluid_mask.ravel())          # x-fastest order
    xs = np.stack([r.x, r.y, r.z], 1)[sc.n_particles:]
    assert len(xs) == len(cells)
    for q, c in enumerate(cells):
        ijk = (c % n, (c // n) % n, c // n ** 2)
        ctr = ((step * n ** 3 + c) * 64 + 1) * 3            # slot 1: the cell held one
        U = S.uniform01(np.array([ctr, ctr + 1, ctr + 2]), 1234)
        want = np.float32((np.array(ijk) + U) * (1 / n)).astype(np.float64)
        assert np.array_equal(xs[q], want), (q, xs[q], want)


def test_hydrostatic_refill_takes_zero_velocity():
    """At rest under gravity the projected interior velocity is exactly zero (the
    hydrostatic closed form), so refilled particles are created at rest."""
    sc = S.layer(16, 8)
    p = O.Params(n=(16, 16, 16), dx=1 / 16, ppc_min=10, cg_tol=1e-13)
    r = O.step(p, *sc.arrays(), fields=False)
    assert r.added == 2 * 16 * 16 * 8
    new = slice(sc.n_particles, None)
    vmax = max(np.abs(r.u[new]).max(), np.abs(r.v[new]).max(), np.abs(r.w[new]).max())
    assert vmax < 1e-10 * 9.81 / 240


def test_over_full_cells_keep_their_lowest_indices():
    n = 8
    sc = S.box(n, (0.25, 0.25, 0.25), (0.75, 0.5, 0.5), density=3)   # 27 per cell
    p = O.Params(n=(n, n, n), dx=1 / n, gravity=(0.0, 0.0, 0.0), ppc_max=12)
    r = O.step(p, *sc.arrays(), fields=False)
    nf = sc.fluid_mask.sum()
    assert r.removed == 15 * nf and len(r.x) == 12 * nf
    c0 = _cells(p, sc.x, sc.y, sc.z)
    keep = np.concatenate([np.flatnonzero(c0 == c)[:12] for c in np.unique(c0)])
    keep.sort()
    assert np.array_equal(r.x, sc.x[keep].astype(np.float64))


def test_capacity_stops_the_refill():
    n = 8
    sc = S.box(n, (0.25, 0.25, 0.25), (0.5, 0.5, 0.5), density=1)
    p = O.Params(n=(n, n, n), dx=1 / n, gravity=(0.0, 0.0, 0.0), ppc_min=3)
    r = O.step(p, *sc.arrays(), fields=False, capacity=sc.n_particles + 5)
    assert r.status == 4 and len(r.x) == sc.n_particles + 5 and r.added == 5
