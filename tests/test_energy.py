"""Energy diagnostic (Sec. 4, Fig. 10): the oracle's sums pinned to hand-computed
values and invariants, the paper's second and third scenes, and the oracle's
energy behaviour over a run (the downward drift Fig. 10 shows)."""
import numpy as np
import pytest

import oracle as O
from paper_2404_01931_gb300 import scenes as S

G = (0.0, -9.81, 0.0)


def test_energy_hand_example():
    # two particles, m = 0.5: |v|^2 = 9 and 25; heights 0.25 and 0.5
    x = np.array([0.1, 0.2]); y = np.array([0.25, 0.5]); z = np.array([0.3, 0.4])
    u = np.array([1.0, 0.0]); v = np.array([2.0, 3.0]); w = np.array([2.0, 4.0])
    ke, pe, tot = O.energy(G, 0.5, x, y, z, u, v, w)
    assert ke == pytest.approx(0.25 * 34.0, rel=1e-15)
    assert pe == pytest.approx(0.5 * 9.81 * 0.75, rel=1e-15)
    assert tot == pytest.approx(ke + pe, rel=1e-15)


def test_energy_invariants():
    sc = S.random_velocities(S.dam_break(16), 0.7, seed=3)
    m = 1.0 / (8 * 16 ** 3)
    ke, pe, _ = O.energy(G, m, *sc.arrays())
    # kinetic: independent of positions and of the sign of the velocities
    ke2, _, _ = O.energy(G, m, sc.x + 0.1, sc.y, sc.z, -sc.u, -sc.v, -sc.w)
    assert ke2 == pytest.approx(ke, rel=1e-14)
    # potential: a shift d of every position adds -m N g . d
    d = np.array([0.01, 0.02, -0.03])
    _, pe2, _ = O.energy(G, m, sc.x + d[0], sc.y + d[1], sc.z + d[2], sc.u, sc.v, sc.w)
    n = sc.n_particles
    assert pe2 - pe == pytest.approx(-m * n * float(np.dot(G, d)), rel=1e-9)
    # linear in the mass, zero for a weightless set at rest
    ke3, pe3, _ = O.energy(G, 2 * m, *sc.arrays())
    assert (ke3, pe3) == (pytest.approx(2 * ke, rel=1e-15), pytest.approx(2 * pe, rel=1e-15))
    assert O.energy((0.0, 0.0, 0.0), m, sc.x, sc.y, sc.z, 0 * sc.u, 0 * sc.v, 0 * sc.w) == (0.0, 0.0, 0.0)


def test_energy_brute_force_sum():
    sc = S.random_velocities(S.water_drop(12), 0.3, seed=5)
    m = 0.125
    ke, pe, _ = O.energy(G, m, *sc.arrays())
    a = [np.asarray(t, np.float64) for t in sc.arrays()]
    ke_ref = sum(0.5 * m * (a[3][i] ** 2 + a[4][i] ** 2 + a[5][i] ** 2) for i in range(a[0].size))
    pe_ref = sum(m * 9.81 * a[1][i] for i in range(a[0].size))
    assert ke == pytest.approx(ke_ref, rel=1e-13)
    assert pe == pytest.approx(pe_ref, rel=1e-13)


def test_second_and_third_scenes():
    n = 32
    dd = S.double_dam_break(n)
    m = dd.fluid_mask
    # two blocks of 6 cells (centres < 0.2 and > 0.8) by 16 cells, mirror images in x
    assert m.sum() == 2 * 6 * 16 * n
    assert np.array_equal(m, m[:, :, ::-1])
    assert dd.n_particles == 8 * m.sum()
    wd = S.water_drop(n)
    cx, cy, cz = S.cell_centres((n, n, n), 1.0 / n)
    r2 = (cx - 0.5) ** 2 + (cy - 0.6) ** 2 + (cz - 0.5) ** 2
    assert np.array_equal(wd.fluid_mask, r2 < 0.04)
    # every particle sits in a seeded cell
    for sc in (dd, wd):
        i = np.floor(sc.x.astype(np.float64) * n).astype(int)
        j = np.floor(sc.y.astype(np.float64) * n).astype(int)
        k = np.floor(sc.z.astype(np.float64) * n).astype(int)
        assert sc.fluid_mask[k, j, i].all()


def test_oracle_energy_decays_over_a_dam_break():
    """Fig. 10: the total energy of the dam break drifts downward step by step.

    With forward-Euler advection of the blended velocity, a particle in free fall
    loses m g^2 dt^2 / 2 per step, and the PIC share and the projection only remove
    kinetic energy, so the total must not rise beyond rounding."""
    n = 16
    sc = S.dam_break(n)
    p = O.Params(n=(n, n, n), dx=1.0 / n)
    m = p.rho * p.dx ** 3 / 8
    arrs = [a.astype(np.float64) for a in sc.arrays()]
    e = [O.energy(p.gravity, m, *arrs)[2]]
    for _ in range(40):
        r = O.step(p, *arrs, fields=False)
        assert r.status == 0
        arrs = [r.x, r.y, r.z, r.u, r.v, r.w]
        e.append(O.energy(p.gravity, m, *arrs)[2])
    e = np.array(e)
    assert np.all(np.diff(e) <= 1e-12 * e[0]), np.diff(e).max()
    assert e[-1] < e[0]
