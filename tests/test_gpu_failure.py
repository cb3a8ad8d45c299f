"""Failure detection without a GPU fault: every device-side wait of the step is
bounded and reports FLIP_E_TIMEOUT, an allocation refused by the caller's allocator
gives FLIP_E_OOM, and a scene whose step fails leaves the other scenes of a batch or
a server untouched.

The waits are made to run out by a limit far below their normal duration (1 ns):
the grid barriers of the solve and G2P's waits for its bulk copies then give up,
the kernels return, and the context stays usable.  No kernel is made to fault.
"""
import ctypes as C

import numpy as np
import pytest

import oracle as O
from paper_2404_01931_gb300 import flip as F
from paper_2404_01931_gb300 import scenes as S

from parity_util import gpu_step, matched, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytestmark = [pytest.mark.gpu, pytest.mark.skip(reason="needs a CUDA GPU")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _by_id(sim):
    return sim.particles(by_id=True)


@pytest.mark.parametrize("mixed", [False, True])
def test_wait_limit_reports_timeout_and_the_handle_recovers(mixed):
    """A 1 ns limit makes the solve's first grid barrier (and G2P's copy waits) give
    up: the step returns FLIP_E_TIMEOUT.  With the default limits restored and the
    particles rewritten, the same handle steps to the oracle's result."""
    n = 32
    sc = S.dam_break(n)
    op, fp = matched(n)
    if mixed:
        fp.precision = F.FLIP_PREC_MIXED_IR
        fp.cg_tol, fp.ir_tol = 1e-3, 1e-8
        op.cg_tol = 1e-11
    ref = O.step(op, *sc.arrays())
    arrays = sc.arrays()
    with F.Simulation(fp, *arrays) as sim:
        sim.set_wait_timeout(1)
        with pytest.raises(F.FlipError) as ei:
            sim.step(1, stats=True)
        assert ei.value.code == F.FLIP_E_TIMEOUT
        # a second timed-out step: still reported, still no fault
        with pytest.raises(F.FlipError) as ei:
            sim.step(1, stats=True)
        assert ei.value.code == F.FLIP_E_TIMEOUT
        sim.set_wait_timeout(0)
        # the timed-out steps left the particles half advanced: put the scene back
        ids = sim.read(F.PID)
        F.flip_write_particles(sim.h, *[np.ascontiguousarray(a[ids]) for a in arrays])
        rc, st = sim.step(1, stats=True)
        assert rc == F.FLIP_OK and st.n_fluid_cells == ref.n_fluid
        x, y, z, u, v, w = _by_id(sim)
        err = np.abs(np.stack([x, y, z]).astype(np.float64)
                     - np.stack([ref.x, ref.y, ref.z])).max() * n
        assert err <= 1e-4, err
        p = sim.read(F.PRESSURE_F64)
        assert rel_l2(p, ref.pressure) <= 1e-5


def test_long_wait_limit_changes_nothing():
    """A limit above the default is only a bound: the step is unchanged."""
    sc = S.dam_break(24)
    op, fp = matched(24)
    ref = O.step(op, *sc.arrays())
    with F.Simulation(fp, *sc.arrays()) as sim:
        sim.set_wait_timeout(20_000_000_000)
        rc, _ = sim.step(1, stats=True)
        assert rc == F.FLIP_OK
        assert rel_l2(sim.read(F.PRESSURE_F64), ref.pressure) <= 1e-5


class _CountingAllocator:
    """A flip_alloc hook over torch's caching allocator that refuses its k-th
    request (returns NULL), counting requests and frees."""

    def __init__(self, fail_at):
        self.fail_at = fail_at
        self.calls = 0
        self.live = {}

        def _alloc(ctx, nbytes, stream):
            self.calls += 1
            if self.calls == self.fail_at:
                return None
            ptr = torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                     int(stream or 0))
            self.live[int(ptr)] = int(nbytes)
            return ptr

        def _free(ctx, ptr, nbytes, stream):
            assert self.live.pop(int(ptr)) == int(nbytes)
            torch.cuda.caching_allocator_delete(int(ptr))

        self._fa = F._ALLOC_FN(_alloc)
        self._ff = F._FREE_FN(_free)
        self.struct = F.FlipAlloc(None, self._fa, self._ff)


def test_refused_allocation_gives_oom_and_leaves_nothing():
    """flip_create takes one arena through the caller's allocator: when the hook
    refuses it the call fails with FLIP_E_OOM and frees nothing it did not get; a
    handle created before keeps working and returns its memory at destroy."""
    sc = S.dam_break(16)
    p = F.default_params(16)
    al = _CountingAllocator(fail_at=2)
    h1, keep1 = F.flip_create(p, *sc.arrays(), allocator=al)
    assert al.calls == 1 and len(al.live) == 1
    with pytest.raises(F.FlipError) as ei:
        F.flip_create(p, *sc.arrays(), allocator=al)
    assert ei.value.code == F.FLIP_E_OOM
    assert al.calls == 2 and len(al.live) == 1
    rc, st = F.flip_step(h1, 1, stats=True)
    assert rc == F.FLIP_OK and st.n_particles == sc.n_particles
    F.flip_destroy(h1)
    assert not al.live
    # the next request succeeds again
    h3, keep3 = F.flip_create(p, *sc.arrays(), allocator=al)
    F.flip_destroy(h3)
    assert not al.live


def _singular_box(n):
    """Every cell fluid: A is singular (no air), the step fails with FLIP_E_ARG."""
    return S.box(n, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), seed=1)


def _check_against_oracle(sim_fields, sc):
    """A scene's step equals the oracle's at the parity bar (pressure and projected
    velocities at relative L2 1e-5, positions within 1e-4 of a cell)."""
    n = sc.n[0]
    op, _ = matched(n)
    ref = O.step(op, *sc.arrays())
    p, u_new, parts = sim_fields
    if p is not None:
        assert rel_l2(p, ref.pressure) <= 1e-5
        fl = 9.81 / 240 * np.sqrt((n + 1) * n * n)
        for d in range(3):
            assert rel_l2(u_new[d], ref.u_new[d], fl) <= 1e-5
    x = np.stack(parts[:3]).astype(np.float64)
    assert np.abs(x - np.stack([ref.x, ref.y, ref.z])).max() * n <= 1e-4


def _fields(sim):
    return (sim.read(F.PRESSURE_F64), [sim.read(f) for f in (F.U_NEW, F.V_NEW, F.W_NEW)],
            sim.particles())


@pytest.mark.parametrize("fused", [False, True])
def test_batch_isolates_a_failing_scene(fused):
    """A scene whose solve is refused (singular: every cell fluid) in a batch, in
    either form: the batch reports FLIP_E_ARG, and the other scenes still equal the
    oracle's step."""
    good = [S.dam_break(24), S.dam_break(32, 0.4, 0.6)]
    bad = _singular_box(16)
    scenes = [good[0], bad, good[1]]
    sims = [F.Simulation(matched(sc.n[0])[1], *sc.arrays()) for sc in scenes]
    try:
        with F.Batch(4) as b:
            b.set_fused(fused)
            with pytest.raises(F.FlipError) as ei:
                b.step(sims, 1, stats=True)
            assert ei.value.code == F.FLIP_E_ARG
        for k in (0, 2):
            _check_against_oracle(_fields(sims[k]), scenes[k])
    finally:
        for s in sims:
            s.close()


def test_server_isolates_a_failing_scene():
    """The same inside the server: the failing scene's request completes with
    FLIP_E_ARG, the others with FLIP_OK and the oracle's particles."""
    good = [S.dam_break(24), S.dam_break(32, 0.4, 0.6)]
    bad = _singular_box(16)
    scenes = [good[0], bad, good[1]]
    with F.Server(8 << 30, 8) as srv:
        ids = [srv.add_scene(matched(sc.n[0])[1], *sc.arrays()) for sc in scenes]
        srv.drain()
        tickets = [srv.submit(i) for i in ids]
        infos = []
        for t in tickets:
            info = F.RequestInfo()
            rc = F.lib().flip_server_wait(srv.s, int(t), C.byref(info))
            infos.append((rc, info.status))
        assert infos[1] == (F.FLIP_E_ARG, F.FLIP_E_ARG)
        assert infos[0] == (F.FLIP_OK, F.FLIP_OK) and infos[2] == (F.FLIP_OK, F.FLIP_OK)
        for k in (0, 2):
            _check_against_oracle((None, None, srv.particles(ids[k])), scenes[k])
