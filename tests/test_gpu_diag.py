"""Energy diagnostic (Sec. 4, Fig. 10) and the paper's other two benchmark scenes on
the CUDA path, against the FP64 oracle, through the C ABI."""
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

G = (0.0, -9.81, 0.0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("trim", [0, 1, 3])
def test_energy_matches_oracle_on_the_same_particles(trim):
    """Same float32 particles on both sides: kinetic and potential energy agree to
    FP64 rounding (float-pair sums on the GPU); ragged counts exercise the tail."""
    sc = S.random_velocities(S.dam_break(48), 0.9, seed=7)
    arrs = [a[: a.size - trim] for a in sc.arrays()]
    fp = matched(48)[1]
    m = 1.0 / (8 * 48 ** 3)
    ref = O.energy(G, m, *arrs)
    with F.Simulation(fp, *arrs) as sim:
        got = sim.energy(m)
    for a, b in zip(got, ref):
        assert a == pytest.approx(b, rel=1e-12, abs=0.0)


def test_energy_of_no_particles_and_argument_checks():
    fp = matched(16)[1]
    e = np.zeros(0, np.float32)
    with F.Simulation(fp, e, e, e, e, e, e) as sim:
        assert sim.energy(1.0) == (0.0, 0.0, 0.0)
        with pytest.raises(F.FlipError):
            sim.energy(-1.0)
        with pytest.raises(F.FlipError):
            sim.energy(float("nan"))


def test_energy_trace_follows_the_oracle():
    """Fig. 10 compares the energy traces of two implementations; here the FP32 CUDA
    path and the FP64 oracle run the 32^3 dam break from the same seeded state, and
    the totals stay within 1e-5 of each other over 10 steps."""
    sc = S.dam_break(32)
    op, fp = matched(32)
    m = op.rho * op.dx ** 3 / 8
    arrs = [a.astype(np.float64) for a in sc.arrays()]
    ref = [O.energy(op.gravity, m, *arrs)]
    for _ in range(10):
        r = O.step(op, *arrs, fields=False)
        arrs = [r.x, r.y, r.z, r.u, r.v, r.w]
        ref.append(O.energy(op.gravity, m, *arrs))
    got = []
    with F.Simulation(fp, *sc.arrays()) as sim:
        got.append(sim.energy(m))
        for _ in range(10):
            sim.step(1)
            got.append(sim.energy(m))
    ref, got = np.array(ref), np.array(got)
    assert got[0] == pytest.approx(ref[0], rel=1e-12)
    err = np.abs(got[:, 2] - ref[:, 2]).max() / ref[0, 2]
    assert err <= 1e-5, err
    kerr = np.abs(got[:, 0] - ref[:, 0]).max() / max(ref[:, 0].max(), 1e-300)
    assert kerr <= 1e-4, kerr


def test_energy_decays_over_200_steps():
    """Fig. 10's setting: a dam break of ~25-33k particles for 200 steps.  The total
    energy drifts down (forward Euler and the PIC share dissipate; nothing adds
    energy), up to FP32 noise per step."""
    sc = S.dam_break(32)
    fp = matched(32)[1]
    m = fp.rho * fp.dx ** 3 / 8
    e = []
    with F.Simulation(fp, *sc.arrays()) as sim:
        e.append(sim.energy(m)[2])
        for _ in range(200):
            assert sim.step(1)[0] == F.FLIP_OK
            e.append(sim.energy(m)[2])
    e = np.array(e)
    assert e[-1] < 0.99 * e[0]
    assert np.diff(e).max() <= 1e-6 * e[0], np.diff(e).max() / e[0]


@pytest.mark.parametrize("scene", ["double_dam_break", "water_drop"])
def test_other_benchmark_scenes_single_step(scene):
    sc = getattr(S, scene)(32)
    op, fp = matched(32)
    ref = O.step(op, *sc.arrays())
    got = gpu_step(fp, sc.arrays())
    assert got["rc"] == F.FLIP_OK
    assert got["stats"].n_fluid_cells == ref.n_fluid
    assert np.array_equal(got["type"].reshape(ref.type.shape), ref.type)
    fl = 9.81 / 240 * np.sqrt(33 * 32 * 32)
    for d in range(3):
        assert rel_l2(got["u_new"][d], ref.u_new[d], fl) <= 1e-5
    assert rel_l2(got["p"], ref.pressure) <= 1e-5
    x, y, z = got["particles"][:3]
    err = max(np.abs(np.asarray(a, np.float64) - b).max() for a, b in ((x, ref.x), (y, ref.y), (z, ref.z)))
    assert err * 32 <= 1e-4
