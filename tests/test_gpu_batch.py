"""Batched scenes: one cooperative solve launch for many uneven scenes.

A scene's results in a batch equal its results alone (up to the order of
floating-point sums: P2G atomics and the per-team reductions), and match the
oracle like a scene stepped alone."""
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


def _mix():
    """Uneven scenes: sizes, a ragged grid, both precisions, both preconditioners."""
    out = []
    for n, mixed, pre in [(32, False, 1), (40, False, 1), (24, True, 1), (48, False, 0),
                          ((20, 13, 17), False, 1), (32, True, 0)]:
        if np.isscalar(n):
            sc = S.random_velocities(S.dam_break(n, 0.4, 0.5, seed=n), 0.2, n)
        else:
            sc = S.random_velocities(S.box(n, (0.0, 0.0, 0.0), (0.55, 0.5, 0.8), seed=5), 0.3, 4)
        op, fp = matched(n, preconditioner=pre)
        if mixed:
            fp.precision = F.FLIP_PREC_MIXED_IR
            fp.cg_tol, fp.ir_tol = 1e-3, 1e-8
        out.append((n, sc, op, fp))
    return out


def _fields(sim):
    return sim.particles() + [sim.read(F.PRESSURE_F64)]


def test_batch_equals_alone():
    """Three steps batched against the same steps alone.  The two runs differ only
    in the order of floating-point sums (P2G atomics, the solver's team reductions),
    but each FP32-mode solve stops at a relative residual of 1e-6, and two solutions
    that both meet that stop can differ by up to kappa(A) * 1e-6 ~ 1e-4 on these
    deep columns; after three steps the particles carry that difference.  Hence
    1e-4 here; each batched scene's single step is held to the 1e-5 parity bar
    against the oracle in test_fused_batch_matches_the_oracle_per_scene."""
    mix = _mix()
    alone = []
    for n, sc, op, fp in mix:
        with F.Simulation(fp, *sc.arrays()) as sim:
            sim.step(3)
            alone.append(_fields(sim))
    sims = [F.Simulation(fp, *sc.arrays()) for n, sc, op, fp in mix]
    try:
        with F.Batch(len(sims)) as b:
            rc, st = b.step(sims, 3, stats=True)
            assert rc == F.FLIP_OK and len(st) == len(sims)
            assert all(s.steps == 3 and s.cg_iterations > 0 for s in st)
        for (n, *_), sim, ref in zip(mix, sims, alone):
            got = _fields(sim)
            dx = 1.0 / (n if np.isscalar(n) else max(n))
            pos = np.abs(np.stack(got[:3]) - np.stack(ref[:3])).max() / dx
            assert pos <= 1e-4, (n, pos)
            assert rel_l2(np.stack(got[3:6]), np.stack(ref[3:6]), 1e-3) <= 1e-4, n
            assert rel_l2(got[6], ref[6]) <= 1e-4, n
    finally:
        for s in sims:
            s.close()


def test_batched_scene_matches_the_oracle():
    n = 32
    sc = S.dam_break(n)
    op, fp = matched(n)
    ref = O.step(op, *sc.arrays())
    other = S.dam_break(40, 0.3, 0.6, seed=9)
    with F.Simulation(fp, *sc.arrays()) as a, \
            F.Simulation(matched(40)[1], *other.arrays()) as o, F.Batch(4) as b:
        rc, _ = b.step([o, a], 1, stats=True)
        assert rc == F.FLIP_OK
        x, y, z, u, v, w = a.particles()
        p = a.read(F.PRESSURE_F64)
    assert np.abs(np.stack([x, y, z]) - np.stack([ref.x, ref.y, ref.z])).max() * n <= 1e-4
    assert rel_l2(p, ref.pressure) <= 1e-5


def test_batch_argument_checks():
    sc = S.dam_break(16)
    fp = matched(16)[1]
    with F.Simulation(fp, *sc.arrays()) as a, F.Batch(2) as b:
        with pytest.raises(F.FlipError) as ei:
            b.step([a, a], 1)
        assert ei.value.code == F.FLIP_E_ARG
        with F.Simulation(fp, *sc.arrays()) as c, F.Simulation(fp, *sc.arrays()) as d:
            with pytest.raises(F.FlipError):
                b.step([a, c, d], 1)  # more than the capacity
        rc, _ = b.step([], 1)
        assert rc == F.FLIP_OK


def test_batch_with_adaptive_step_and_reseeding():
    """Scenes with the adaptive time step and reseeding in one batch: each takes the
    dt, particle count and per-cell counts it takes alone."""
    specs = [(24, 3.0, (3, 12)), (32, 0.0, (3, 0)), (16, 0.01, (0, 6))]
    scenes, params = [], []
    for n, cfl, (lo, hi) in specs:
        sc = S.random_velocities(S.box(n, (0.1, 0.0, 0.1), (0.7, 0.6, 0.8), density=1, seed=n), 20.0, n)
        fp = matched(n)[1]
        fp.cfl, fp.ppc_min, fp.ppc_max = cfl, lo, hi
        fp.max_particles = 40 * sc.n_particles   # fast lone particles spread into many cells
        scenes.append(sc)
        params.append(fp)

    def cells(n, sim):
        x, y, z = (sim.read(f).astype(np.float64) for f in (F.PX, F.PY, F.PZ))
        c = lambda a: np.clip(np.floor(a * n).astype(int), 0, n - 1)
        return np.bincount(c(x) + n * (c(y) + n * c(z)), minlength=n ** 3)

    alone = []
    for (n, _, _), sc, fp in zip(specs, scenes, params):
        with F.Simulation(fp, *sc.arrays()) as sim:
            rc, st = sim.step(3, stats=True)
            assert rc == F.FLIP_OK
            alone.append((st.dt_last, st.n_particles, cells(n, sim)))
    sims = [F.Simulation(fp, *sc.arrays()) for sc, fp in zip(scenes, params)]
    try:
        with F.Batch(len(sims)) as b:
            rc, sts = b.step(sims, 3, stats=True)
        assert rc == F.FLIP_OK
        for (n, _, _), sim, st, (dt, npart, cnt) in zip(specs, sims, sts, alone):
            assert st.dt_last == pytest.approx(dt, rel=1e-6)
            assert st.n_particles == npart
            # a particle that ends a step within rounding of a cell face may land on
            # either side in the two runs (their sums differ in order): one cell one
            # less, its neighbour one more
            assert np.abs(cells(n, sim) - cnt).sum() <= 2
    finally:
        for s in sims:
            s.close()


def test_autotune_picks_a_candidate_and_keeps_results():
    """The autotuner advances the scenes by real steps (2 x 7 for the split, 2 x 4 x
    (2 + 2) for the forms, 2 x 3 for the transfers' launch shapes) and leaves a
    split, a form and launch shapes in force; from the initial particles again, the
    scenes then step as they do alone (these change only the order of
    floating-point sums)."""
    mix = _mix()[:4]
    sims = [F.Simulation(fp, *sc.arrays()) for n, sc, op, fp in mix]
    ref = []
    for n, sc, op, fp in mix:
        with F.Simulation(fp, *sc.arrays()) as sim:
            sim.step(2)
            ref.append(sim.read(F.PRESSURE_F64))
    try:
        with F.Batch(len(sims)) as b:
            a = b.autotune(sims, 1)
            assert a in (0.5, 0.75, 1.0, 1.25, 1.5, 2.0, 2.5)
            assert b.form() in ((True, False), (True, True), (False, False), (False, True))
            shapes = {sim.transfer_ctas() for sim in sims}
            assert len(shapes) == 1                 # the same shapes on every scene
            p2g, g2p = shapes.pop()
            assert p2g in (4, 8, 16) and g2p >= 1
            # the autotuner took 14 + 8 * 4 + 6 = 52 steps; start the scenes again
            for sim, (n, sc, op, fp) in zip(sims, mix):
                ids = sim.read(F.PID)
                F.flip_write_particles(sim.h, *[np.ascontiguousarray(x[ids]) for x in sc.arrays()])
            rc, st = b.step(sims, 2, stats=True)
            assert rc == F.FLIP_OK
            for sim, p in zip(sims, ref):
                assert rel_l2(sim.read(F.PRESSURE_F64), p) <= 1e-4
        with F.Batch(2) as b2:
            with pytest.raises(F.FlipError):
                b2.set_team_exponent(-1.0)
    finally:
        for s_ in sims:
            s_.close()


def test_graph_replay_equals_plain_steps():
    """Pairs of batched steps replayed as a captured CUDA graph give the results of
    the same steps launched one by one (up to the order of floating-point sums).
    One solver group (FP32, multigrid): batches of several groups keep the plain
    path."""
    mix = [m for m in _mix() if m[3].precision == F.FLIP_PREC_FP32 and m[3].preconditioner == 1]
    assert len(mix) >= 3
    plain, graph = [], []
    for store, use in ((plain, False), (graph, True)):
        sims = [F.Simulation(fp, *sc.arrays()) for n, sc, op, fp in mix]
        try:
            with F.Batch(len(sims)) as b:
                b.set_graphs(use)
                b.step(sims, 5)                  # two captured pairs and one plain step
                b.step(sims, 4)                  # the cached graph, twice
                assert b.graph_active() == use
                for s in sims:
                    store.append(_fields(s))
        finally:
            for s in sims:
                s.close()
    for a, b_ in zip(plain, graph):
        for x, y in zip(a, b_):
            assert rel_l2(y, x, 1e-3) <= 1e-4


def test_batch_with_a_gauss_seidel_scene():
    """A scene using the red-black Gauss-Seidel solver shares the batched launch of
    the multigrid scenes and takes the same pressure it takes alone."""
    sc1 = S.dam_break(24, 0.4, 0.5)
    sc2 = S.dam_break(32, 0.4, 0.5, seed=2)
    fp1 = matched(24, preconditioner=F.FLIP_PRECOND_RBGS, cg_max_iter=5000, cg_tol=1e-4)[1]
    fp2 = matched(32)[1]
    alone = []
    for fp, sc in ((fp1, sc1), (fp2, sc2)):
        with F.Simulation(fp, *sc.arrays()) as sim:
            sim.step(2)
            alone.append(sim.read(F.PRESSURE_F64))
    sims = [F.Simulation(fp1, *sc1.arrays()), F.Simulation(fp2, *sc2.arrays())]
    try:
        with F.Batch(2) as b:
            rc, st = b.step(sims, 2, stats=True)
            assert rc == F.FLIP_OK
        for s, p in zip(sims, alone):
            assert rel_l2(s.read(F.PRESSURE_F64), p) <= 1e-4
    finally:
        for s in sims:
            s.close()


def test_fused_batch_matches_the_oracle_per_scene():
    """The fused form (one launch per step kernel for all scenes): every scene of an
    uneven mix -- sizes, a ragged grid, both precisions, both preconditioners --
    matches the FP64 oracle's step at the parity bar: pressure and projected
    velocities at relative L2 1e-5, positions within 1e-4 of a cell."""
    mix = _mix()
    sims = [F.Simulation(fp, *sc.arrays()) for n, sc, op, fp in mix]
    try:
        with F.Batch(len(sims)) as b:
            b.set_fused(True)
            rc, st = b.step(sims, 1, stats=True)
            assert rc == F.FLIP_OK
            # one launch per kernel for all scenes, not ~8 per scene: 7 for the binning,
            # P2G and right-hand side, one solve per (precision, preconditioner) group
            # (4 here), one G2P per precision (2), and scene 0's statistics kernel
            assert st[0].kernel_launches == 7 + 4 + 2 + 1, st[0].kernel_launches
        for (n, sc, op, fp), sim in zip(mix, sims):
            if fp.precision == F.FLIP_PREC_MIXED_IR:
                op.cg_tol, op.cg_max_iter = 1e-11, 100000
            ref = O.step(op, *sc.arrays())
            nn = (n, n, n) if np.isscalar(n) else n
            m = max(nn)
            assert rel_l2(sim.read(F.PRESSURE_F64), ref.pressure) <= 1e-5, n
            fl = 9.81 / 240 * np.sqrt((nn[0] + 1) * nn[1] * nn[2])
            for d, f in enumerate((F.U_NEW, F.V_NEW, F.W_NEW)):
                assert rel_l2(sim.read(f), ref.u_new[d], fl) <= 1e-5, (n, d)
            x, y, z, u, v, w = sim.particles()
            err = np.abs(np.stack([x, y, z]).astype(np.float64)
                         - np.stack([ref.x, ref.y, ref.z])).max() * m
            assert err <= 1e-4, (n, err)
    finally:
        for s in sims:
            s.close()


def test_fused_and_per_scene_forms_agree():
    """The fused form and the per-scene launches compute the same steps (up to the
    order of floating-point sums), over three steps and with the CUDA-graph replay."""
    mix = [m for m in _mix() if m[3].precision == F.FLIP_PREC_FP32 and m[3].preconditioner == 1]
    out = {}
    for fused, graphs in ((False, False), (True, False), (True, True)):
        sims = [F.Simulation(fp, *sc.arrays()) for n, sc, op, fp in mix]
        try:
            with F.Batch(len(sims)) as b:
                b.set_fused(fused)
                b.set_graphs(graphs)
                b.step(sims, 3)
                out[(fused, graphs)] = [_fields(s) for s in sims]
                assert b.graph_active() == graphs
        finally:
            for s in sims:
                s.close()
    base = out[(False, False)]
    for key in ((True, False), (True, True)):
        for a, c in zip(base, out[key]):
            for x, y in zip(a, c):
                assert rel_l2(y, x, 1e-3) <= 1e-4, key


def test_fused_batch_edge_scenes():
    """The fused form over degenerate and many scenes: an empty scene, a one-particle
    scene, grids smaller than a brick and not a multiple of it, and 300 small scenes in
    one call (the binary search over the CTA ranges and the flat brick list).  Every
    non-empty scene matches the oracle's step; the empty one stays empty."""
    specs = [S.dam_break(16), S.box((4, 5, 6), (0.0, 0.0, 0.0), (0.5, 0.6, 1.0), seed=2),
             S.box((9, 17, 11), (0.1, 0.0, 0.2), (0.8, 0.4, 0.9), seed=3)]
    one = S.box(8, (0.0, 0.0, 0.0), (0.125, 0.125, 0.125), density=1, seed=4)
    assert one.n_particles == 1
    specs.append(one)
    specs += [S.dam_break(8, 0.5, 0.5, seed=10 + k) for k in range(296)]
    empty = np.zeros(0, np.float32)
    sims = [F.Simulation(matched(8)[1], empty, empty, empty, empty, empty, empty)]
    sims += [F.Simulation(matched(sc.n)[1], *sc.arrays()) for sc in specs]
    try:
        with F.Batch(len(sims)) as b:
            b.set_fused(True)
            rc, st = b.step(sims, 1, stats=True)
            assert rc == F.FLIP_OK
        assert st[0].n_particles == 0 and st[0].n_fluid_cells == 0
        for k in (1, 2, 3, 4, 5, 150, 299):
            sc, sim = specs[k - 1], sims[k]
            op = matched(sc.n)[0]
            ref = O.step(op, *sc.arrays())
            x, y, z, u, v, w = sim.particles()
            err = np.abs(np.stack([x, y, z]).astype(np.float64)
                         - np.stack([ref.x, ref.y, ref.z])).max() * max(sc.n)
            assert err <= 1e-4, (k, err)
            assert rel_l2(sim.read(F.PRESSURE_F64), ref.pressure) <= 1e-5, k
    finally:
        for s_ in sims:
            s_.close()
