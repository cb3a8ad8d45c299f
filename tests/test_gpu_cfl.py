"""Adaptive time step (Sec. 3.1.4) on the CUDA path against the FP64 oracle.

The GPU takes dt from the largest particle speed the previous G2P (or the
creation) recorded and solves for q = dt p / (rho dx^2); reads return p.  Both
sides must take the same dt (to FP32 rounding of the speeds) and the same fields."""
import numpy as np
import pytest

import oracle as O
from paper_2404_01931_gb300 import flip as F
from paper_2404_01931_gb300 import scenes as S

from parity_util import face_floor, gpu_step, matched, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytestmark = [pytest.mark.gpu, pytest.mark.skip(reason="needs a CUDA GPU")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _fields_match(ref, got, n, tol=1e-5):
    fl = face_floor(n)
    assert np.array_equal(got["type"].reshape(ref.type.shape), ref.type)
    for d in range(3):
        assert rel_l2(got["u_old"][d], ref.u_old[d], fl) <= tol
        assert rel_l2(got["u_new"][d], ref.u_new[d], fl) <= tol
    assert rel_l2(got["rhs"], ref.rhs) <= tol
    assert rel_l2(got["p"], ref.pressure) <= tol


@pytest.mark.parametrize("mixed", [False, True])
def test_cfl_single_step_matches_the_oracle(mixed):
    n = 24
    sc = S.random_velocities(S.box(n, (0.1, 0.0, 0.2), (0.7, 0.55, 0.9), seed=11), 40.0, 3)
    op, fp = matched(n, cg_tol=1e-12 if mixed else 1e-6)
    op.cfl = fp.cfl = 3.0
    ref = O.step(op, *sc.arrays())
    assert ref.dt < op.dt                              # the limit is active
    if mixed:
        fp.cg_tol, fp.ir_tol = 0.1, 1e-9
    got = gpu_step(fp, sc.arrays(), precision=F.FLIP_PREC_MIXED_IR if mixed else None)
    assert got["stats"].dt_last == pytest.approx(ref.dt, rel=1e-6)
    _fields_match(ref, got, n)
    x, y, z = got["particles"][:3]
    err = max(np.abs(np.asarray(a, np.float64) - b).max() for a, b in ((x, ref.x), (y, ref.y), (z, ref.z)))
    assert err * n <= 1e-4


def test_cfl_trajectory_follows_the_oracle():
    """Ten free-running steps of the 32^3 dam break with a CFL number small enough to
    bind from the second step on: per-step dt and final positions match."""
    n = 32
    sc = S.dam_break(n)
    op, fp = matched(n)
    op.cfl = fp.cfl = 0.003
    arrs = [a.astype(np.float64) for a in sc.arrays()]
    ref_dt = []
    for _ in range(10):
        r = O.step(op, *arrs, fields=False)
        ref_dt.append(r.dt)
        arrs = [r.x, r.y, r.z, r.u, r.v, r.w]
    got_dt = []
    with F.Simulation(fp, *sc.arrays()) as sim:
        for _ in range(10):
            rc, st = sim.step(1, stats=True)
            assert rc == F.FLIP_OK
            got_dt.append(st.dt_last)
        parts = sim.particles()
    assert ref_dt[0] == op.dt and min(ref_dt[1:]) < op.dt
    assert np.allclose(got_dt, ref_dt, rtol=1e-5, atol=0.0)
    err = max(np.abs(np.asarray(parts[a], np.float64) - arrs[a]).max() for a in range(3))
    assert err * n <= 1e-4


def test_cfl_at_rest_takes_dt_max():
    sc = S.layer(32, 16)
    op, fp = matched(32)
    fp.cfl = 3.0
    got = gpu_step(fp, sc.arrays(), nsteps=2)
    assert got["stats"].dt_last == fp.dt
