"""The CUDA path against the counts and constants the paper states
(tests/golden/paper_facts.txt), beside the oracle on the same inputs."""
import numpy as np
import pytest

import oracle as O
from paper_2404_01931_gb300 import flip as F
from paper_2404_01931_gb300 import scenes as S

from parity_util import matched
from test_golden import facts

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytestmark = [pytest.mark.gpu, pytest.mark.skip(reason="needs a CUDA GPU")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _counts(n, x, y, z):
    c = np.clip(np.floor(np.stack([x, y, z], 1).astype(np.float64) * n), 0, n - 1).astype(np.int64)
    return np.bincount(c @ np.array([1, n, n * n]), minlength=n ** 3)


def test_reseeding_bounds():
    """One step of a still, weightless scene of one-particle and 27-particle cells:
    every non-empty cell ends with 3 to 12 particles, as in the oracle."""
    f = facts()
    lo, hi = f["reseed_min_per_cell"], f["reseed_max_per_cell"]
    n = 16
    a = S.box(n, (0.1, 0.1, 0.1), (0.4, 0.4, 0.4), density=1)
    b = S.box(n, (0.6, 0.6, 0.6), (0.9, 0.9, 0.9), density=3)
    arrs = [np.concatenate([p, q]) for p, q in zip(a.arrays(), b.arrays())]
    op, fp = matched(n, gravity=(0.0, 0.0, 0.0))
    op.ppc_min = fp.ppc_min = lo
    op.ppc_max = fp.ppc_max = hi
    ref = O.step(op, *arrs, fields=False)
    with F.Simulation(fp, *arrs) as sim:
        rc, st = sim.step(1, stats=True)
        assert rc == F.FLIP_OK
        x, y, z = sim.read(F.PX), sim.read(F.PY), sim.read(F.PZ)
    cg = _counts(n, x, y, z)
    assert cg[cg > 0].min() == lo and cg.max() == hi
    assert np.array_equal(cg, _counts(n, ref.x, ref.y, ref.z))
    assert st.particles_added == ref.added and st.particles_removed == ref.removed


def test_cfl_number():
    f = facts()
    n = 32
    sc = S.box(n, (0.3, 0.3, 0.3), (0.6, 0.6, 0.6), velocity=(0.0, 0.0, 50.0))
    op, fp = matched(n)
    op.cfl = fp.cfl = float(f["cfl_alpha"])
    ref = O.step(op, *sc.arrays(), fields=False)
    assert ref.dt == f["cfl_alpha"] * (1.0 / n) / 50.0
    with F.Simulation(fp, *sc.arrays()) as sim:
        rc, st = sim.step(1, stats=True)
        assert rc == F.FLIP_OK
    assert st.dt_last == pytest.approx(ref.dt, rel=1e-6)
