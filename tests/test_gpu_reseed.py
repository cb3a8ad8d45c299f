"""Reseeding (Sec. 3.1.2) on the CUDA path against the FP64 oracle.

Unique results are compared exactly: particle counts per cell, and the new
particles' positions (the same SplitMix64 counter and float rounding on both
sides).  The new particles' order in the buffer and their ids come from an atomic
on the GPU, so new particles are matched as sets (by position); their velocities
(the projected grid velocity at the position) agree to FP32 rounding.  Which
particles an over-full cell drops is unspecified: the survivors must be a subset
of the cell's particles, with the right count."""
import numpy as np
import pytest

import oracle as O
from paper_2404_01931_gb300 import flip as F
from paper_2404_01931_gb300 import scenes as S

from parity_util import matched, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytestmark = [pytest.mark.gpu, pytest.mark.skip(reason="needs a CUDA GPU")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _cells(n, x, y, z):
    i = np.clip(np.floor(np.asarray(x, np.float64) * n).astype(int), 0, n - 1)
    j = np.clip(np.floor(np.asarray(y, np.float64) * n).astype(int), 0, n - 1)
    k = np.clip(np.floor(np.asarray(z, np.float64) * n).astype(int), 0, n - 1)
    return i + n * (j + n * k)


def _read(sim):
    arrs = [sim.read(f) for f in (F.PX, F.PY, F.PZ, F.PU, F.PV, F.PW)]
    return arrs, sim.read(F.PID)


def _split(arrs, ids, np0):
    old = ids < np0
    order = np.argsort(ids[old])
    o = [a[old][order] for a in arrs]
    new = [a[~old] for a in arrs]
    return o, new


def _sorted_by_position(a):
    key = np.lexsort((a[2], a[1], a[0]))
    return [t[key] for t in a]


@pytest.mark.parametrize("mixed", [False, True])
def test_refill_single_step_matches_the_oracle(mixed):
    n = 24
    sc = S.random_velocities(S.box(n, (0.1, 0.0, 0.1), (0.8, 0.6, 0.9), density=1, seed=2), 0.6, 7)
    op, fp = matched(n, cg_tol=1e-12 if mixed else 1e-6)
    op.ppc_min = fp.ppc_min = 3
    op.reseed_seed = fp.reseed_seed = 77
    ref = O.step(op, *sc.arrays(), fields=False, step_index=0)
    if mixed:
        fp.precision, fp.cg_tol, fp.ir_tol = F.FLIP_PREC_MIXED_IR, 0.1, 1e-9
    np0 = sc.n_particles
    with F.Simulation(fp, *sc.arrays()) as sim:
        rc, st = sim.step(1, stats=True)
        assert rc == F.FLIP_OK
        arrs, ids = _read(sim)
    assert st.particles_added == ref.added > 0 and st.n_particles == len(ref.x)
    assert np.array_equal(np.sort(ids), np.arange(len(ids)))
    # counts per cell
    cg = np.bincount(_cells(n, *arrs[:3]), minlength=n ** 3)
    cr = np.bincount(_cells(n, ref.x, ref.y, ref.z), minlength=n ** 3)
    assert np.array_equal(cg, cr)
    assert cg[cg > 0].min() >= 3
    old, new = _split(arrs, ids, np0)
    # the particles that were there: as in every step
    dpos = max(np.abs(old[a].astype(np.float64) - ref_a[:np0]).max()
               for a, ref_a in enumerate((ref.x, ref.y, ref.z)))
    assert dpos * n <= 1e-4
    vfloor = 9.81 / 240 * np.sqrt(3 * np0)
    assert rel_l2(np.stack(old[3:]), np.stack([ref.u[:np0], ref.v[:np0], ref.w[:np0]]), vfloor) <= 1e-5
    # the new ones: same positions exactly, velocities to FP32 rounding
    gn = _sorted_by_position([t.astype(np.float64) for t in new])
    rn = _sorted_by_position([t[np0:] for t in (ref.x, ref.y, ref.z, ref.u, ref.v, ref.w)])
    for a in range(3):
        assert np.array_equal(gn[a], rn[a])
    assert rel_l2(np.stack(gn[3:]), np.stack(rn[3:]), vfloor) <= 1e-5


def test_refill_with_adaptive_step_over_two_steps():
    n = 24
    sc = S.random_velocities(S.box(n, (0.1, 0.0, 0.1), (0.8, 0.6, 0.9), density=1, seed=2), 30.0, 7)
    op, fp = matched(n)
    op.ppc_min = fp.ppc_min = 3
    op.cfl = fp.cfl = 3.0
    r1 = O.step(op, *sc.arrays(), fields=False, step_index=0)
    r2 = O.step(op, r1.x, r1.y, r1.z, r1.u, r1.v, r1.w, fields=False, step_index=1)
    with F.Simulation(fp, *sc.arrays()) as sim:
        sim.step(1)
        rc, st = sim.step(1, stats=True)
        arrs, _ = _read(sim)
    assert r2.dt < op.dt
    assert st.dt_last == pytest.approx(r2.dt, rel=1e-5)
    cg = np.bincount(_cells(n, *arrs[:3]), minlength=n ** 3)
    cr = np.bincount(_cells(n, r2.x, r2.y, r2.z), minlength=n ** 3)
    assert np.abs(cg - cr).sum() <= 2      # a particle within rounding of a cell face may differ


def test_over_full_cells_are_trimmed():
    n = 16
    sc = S.box(n, (0.25, 0.25, 0.25), (0.75, 0.5, 0.5), density=3)    # 27 per cell, at rest
    op, fp = matched(n, gravity=(0.0, 0.0, 0.0))
    fp.ppc_max = 12
    np0 = sc.n_particles
    with F.Simulation(fp, *sc.arrays()) as sim:
        rc, st = sim.step(1, stats=True)
        arrs, ids = _read(sim)
    nf = sc.fluid_mask.sum()
    assert st.particles_removed == 15 * nf and st.n_particles == 12 * nf == len(ids)
    cg = np.bincount(_cells(n, *arrs[:3]), minlength=n ** 3)
    assert set(np.unique(cg)) == {0, 12}
    # survivors are original particles, unmoved, each once
    assert len(np.unique(ids)) == len(ids) and ids.max() < np0
    assert np.array_equal(arrs[0], sc.x[ids]) and np.array_equal(arrs[1], sc.y[ids])


def test_dam_break_keeps_every_fluid_cell_filled():
    n = 32
    sc = S.dam_break(n)
    fp = matched(n)[1]
    fp.ppc_min, fp.ppc_max = 3, 12
    with F.Simulation(fp, *sc.arrays()) as sim:
        total_add = total_rm = 0
        for _ in range(30):
            rc, st = sim.step(1, stats=True)
            assert rc == F.FLIP_OK
            total_add += st.particles_added
            total_rm += st.particles_removed
            arrs, ids = _read(sim)
            c = np.bincount(_cells(n, *arrs[:3]), minlength=n ** 3)
            assert c[c > 0].min() >= 3
            assert len(np.unique(ids)) == len(ids) == st.n_particles
        e = sim.energy(1.0 / (8 * n ** 3))
    assert total_add > 0
    assert np.isfinite(e[2])
    assert st.n_particles == sc.n_particles + total_add - total_rm


def test_capacity_limit_is_a_warning():
    n = 16
    sc = S.box(n, (0.25, 0.25, 0.25), (0.5, 0.5, 0.5), density=1)
    fp = matched(n, gravity=(0.0, 0.0, 0.0))[1]
    fp.ppc_min = 3
    fp.max_particles = sc.n_particles + 10
    with F.Simulation(fp, *sc.arrays()) as sim:
        with pytest.warns(RuntimeWarning):
            rc, st = sim.step(1, stats=True)
        assert rc == F.FLIP_E_CAPACITY
        assert st.n_particles == sc.n_particles + 10 and st.particles_added == 10
        arrs, ids = _read(sim)
        assert len(ids) == sc.n_particles + 10 and len(np.unique(ids)) == len(ids)
        with pytest.warns(RuntimeWarning):
            rc, st = sim.step(1, stats=True)
        assert st.n_particles == sc.n_particles + 10


def test_reseed_argument_checks():
    sc = S.box(8, (0.25, 0.25, 0.25), (0.5, 0.5, 0.5))
    for field, value in (("ppc_min", 65), ("ppc_min", -1), ("ppc_max", -2)):
        fp = matched(8)[1]
        setattr(fp, field, value)
        with pytest.raises(F.FlipError):
            F.Simulation(fp, *sc.arrays())
    fp = matched(8)[1]
    fp.ppc_min, fp.ppc_max = 5, 3
    with pytest.raises(F.FlipError):
        F.Simulation(fp, *sc.arrays())
    fp = matched(8)[1]
    fp.max_particles = 3
    with pytest.raises(F.FlipError):
        F.Simulation(fp, *sc.arrays())
