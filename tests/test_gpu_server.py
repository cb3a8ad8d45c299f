"""The continuous-batching server: a scene's results are the same served amid other
scenes' requests as stepped alone; scenes are admitted by footprint within the
budget; requests arriving while a batch runs join later batches."""
import numpy as np
import pytest

from paper_2404_01931_gb300 import flip as F
from paper_2404_01931_gb300 import scenes as S

from parity_util import matched

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytestmark = [pytest.mark.gpu, pytest.mark.skip(reason="needs a CUDA GPU")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _scene(n, seed, mixed=False):
    sc = S.random_velocities(S.dam_break(n, 0.45, 0.5, seed=seed), 0.2, seed)
    fp = matched(n)[1]
    if mixed:
        fp.precision = F.FLIP_PREC_MIXED_IR
        fp.cg_tol, fp.ir_tol = 1e-3, 1e-8
    return sc, fp


def test_served_scene_equals_alone():
    """Three steps per scene served amid the others against the same steps alone, at
    the tolerance of test_batch_equals_alone (two FP32 solves that both stop at a
    relative residual of 1e-6 can differ by kappa(A) * 1e-6 ~ 1e-4); each served
    step is held to the parity bar against the oracle in
    test_served_scenes_match_the_oracle."""
    scenes = [_scene(32, 1), _scene(40, 2, mixed=True), _scene(24, 3), _scene(48, 4)]
    alone = []
    for sc, fp in scenes:
        with F.Simulation(fp, *sc.arrays()) as sim:
            sim.step(3)
            alone.append(sim.particles())
    with F.Server(budget_bytes=8 << 30, max_batch=8) as srv:
        ids = [srv.add_scene(fp, *sc.arrays()) for sc, fp in scenes]
        t0 = srv.now() + 0.05
        rng = np.random.default_rng(0)
        tickets = []
        # three steps per scene, interleaved, arriving over ~30 ms
        order = [i for i in ids for _ in range(3)]
        rng.shuffle(order)
        for k, sid in enumerate(order):
            tickets.append(srv.submit(sid, t0 + 0.0025 * k))
        infos = [srv.wait(t) for t in tickets]
        assert all(i.status == F.FLIP_OK for i in infos)
        assert all(i.t_arrival <= i.t_start + 1e-9 and i.t_start <= i.t_done for i in infos)
        for sid, (sc, fp), ref in zip(ids, scenes, alone):
            got = srv.particles(sid)
            dx = 1.0 / sc.n[0]
            assert np.abs(np.stack(got[:3]) - np.stack(ref[:3])).max() / dx <= 1e-4
            assert np.abs(np.stack(got[3:]) - np.stack(ref[3:])).max() <= 1e-4


def test_requests_arriving_together_share_a_batch():
    scenes = [_scene(24, s) for s in range(6)]
    with F.Server(budget_bytes=8 << 30, max_batch=16) as srv:
        ids = [srv.add_scene(fp, *sc.arrays()) for sc, fp in scenes]
        srv.drain()
        t = srv.now() + 0.05
        tickets = [srv.submit(i, t) for i in ids]
        infos = [srv.wait(k) for k in tickets]
        assert max(i.batch_size for i in infos) > 1
        assert all(i.t_done >= t for i in infos)


def test_admission_by_footprint():
    (sa, fa), (sb, fb) = _scene(32, 5), _scene(32, 6)
    need = F.flip_footprint_bytes(fa, sa.n_particles)
    assert need > 0
    with F.Server(budget_bytes=int(need * 1.5), max_batch=4) as srv:
        a = srv.add_scene(fa, *sa.arrays())
        b = srv.add_scene(fb, *sb.arrays())
        ta = srv.submit(a)
        assert srv.wait(ta).status == F.FLIP_OK
        assert srv.usage()[0] == 1           # b does not fit next to a
        tb = srv.submit(b)                   # waits for memory
        srv.remove_scene(a)                  # frees a's memory: b is admitted
        info = srv.wait(tb)
        assert info.status == F.FLIP_OK and srv.usage()[0] == 1
        big, fbig = _scene(64, 7)
        with pytest.raises(F.FlipError) as ei:
            srv.add_scene(fbig, *big.arrays())
        assert ei.value.code == F.FLIP_E_OOM


def test_served_scenes_match_the_oracle():
    """Each scene's served step equals the FP64 oracle's step from the same input at
    the parity bar (positions within 1e-4 of a cell, velocities at relative L2 1e-5),
    in a mix of scene sizes and precisions served as several overlapping batches."""
    import oracle as O
    from parity_util import rel_l2
    scenes = [_scene(32, 11), _scene(40, 12, mixed=True), _scene(24, 13), _scene(48, 14)]
    refs = []
    for sc, fp in scenes:
        op = matched(sc.n[0])[0]
        if fp.precision == F.FLIP_PREC_MIXED_IR:
            op.cg_tol, op.cg_max_iter = 1e-11, 100000
        refs.append(O.step(op, *sc.arrays()))
    with F.Server(budget_bytes=8 << 30, max_batch=2) as srv:
        ids = [srv.add_scene(fp, *sc.arrays()) for sc, fp in scenes]
        srv.drain()
        t0 = srv.now() + 0.02
        tickets = [srv.submit(sid, t0 + 0.001 * k) for k, sid in enumerate(ids)]
        infos = [srv.wait(t) for t in tickets]
        assert all(i.status == F.FLIP_OK for i in infos)
        for sid, (sc, fp), ref in zip(ids, scenes, refs):
            x, y, z, u, v, w = srv.particles(sid)
            n = sc.n[0]
            err = np.abs(np.stack([x, y, z]).astype(np.float64)
                         - np.stack([ref.x, ref.y, ref.z])).max() * n
            assert err <= 1e-4, (n, err)
            vel = np.stack([u, v, w])
            e = rel_l2(vel, np.stack([ref.u, ref.v, ref.w]), 9.81 / 240 * np.sqrt(vel.size))
            assert e <= 1e-5, (n, e)


def test_next_batch_is_enqueued_while_one_runs():
    """With one scene per batch, the second batch is formed and enqueued as soon as the
    first batch's solve is done, while the first scene's G2P (13 M particles) still
    runs: its start precedes the first scene's completion.  Every request completes
    with its own scene's step."""
    big = S.dam_break(128, 0.9, 0.9, seed=30)
    scenes = [(big, matched(128)[1])] + [_scene(32, 31 + k) for k in range(3)]
    with F.Server(budget_bytes=32 << 30, max_batch=1) as srv:
        ids = [srv.add_scene(fp, *sc.arrays()) for sc, fp in scenes]
        srv.drain()
        for _ in range(2):  # warm the kernels and the events
            for t in [srv.submit(i) for i in ids]:
                srv.wait(t)
        t = srv.now() + 0.01
        tickets = [srv.submit(i, t) for i in ids]
        infos = [srv.wait(k) for k in tickets]
        assert all(i.status == F.FLIP_OK and i.batch_size == 1 for i in infos)
        first = min(infos, key=lambda i: i.t_start)
        second = min((i for i in infos if i is not first), key=lambda i: i.t_start)
        assert first.scene == ids[0]
        assert second.t_start < first.t_done, (second.t_start, first.t_done)
