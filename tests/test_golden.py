"""The oracle and the seeded scene generator against the counts and constants the
paper states (tests/golden/paper_facts.txt: value and passage per line)."""
import os

import numpy as np

import oracle as O
from paper_2404_01931_gb300 import scenes as S

HERE = os.path.dirname(os.path.abspath(__file__))


def facts():
    out = {}
    for line in open(os.path.join(HERE, "golden", "paper_facts.txt")):
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        kv, cite = line.split("|", 1)
        k, v = (s.strip() for s in kv.split("="))
        assert cite.strip().startswith("Sec."), line
        out[k] = int(v)
    return out


def test_fixture_is_complete():
    assert set(facts()) == {"seed_subcells_per_axis", "seed_particles_per_cell",
                            "reseed_min_per_cell", "reseed_max_per_cell", "cfl_alpha",
                            "mc_configurations", "mc_trivial_configurations"}


def test_seeding_one_particle_per_subcell():
    f = facts()
    s, n = f["seed_subcells_per_axis"], 16
    sc = S.dam_break(n, 0.25, 0.5, density=s, seed=7)
    assert sc.n_particles == f["seed_particles_per_cell"] * int(sc.fluid_mask.sum())
    sub = np.floor(np.stack([sc.x, sc.y, sc.z], 1).astype(np.float64) * n * s).astype(np.int64)
    key = sub[:, 0] + n * s * (sub[:, 1] + n * s * sub[:, 2])
    assert np.unique(key).size == sc.n_particles        # no subcell holds two
    cell = (sub // s) @ np.array([1, n, n * n])
    counts = np.bincount(cell, minlength=n ** 3)
    assert set(np.unique(counts[counts > 0])) == {f["seed_particles_per_cell"]}


def test_reseeding_keeps_cells_within_the_bounds():
    """A still, weightless scene of one-particle cells and 27-particle cells: one step
    trims the full cells at binning and refills the sparse ones after G2P."""
    f = facts()
    lo, hi = f["reseed_min_per_cell"], f["reseed_max_per_cell"]
    n = 16
    a = S.box(n, (0.1, 0.1, 0.1), (0.4, 0.4, 0.4), density=1)
    b = S.box(n, (0.6, 0.6, 0.6), (0.9, 0.9, 0.9), density=3)
    arrs = [np.concatenate([p, q]) for p, q in zip(a.arrays(), b.arrays())]
    p = O.Params(n=(n, n, n), dx=1 / n, gravity=(0.0, 0.0, 0.0), ppc_min=lo, ppc_max=hi)
    r = O.step(p, *arrs, fields=False)
    assert r.status == 0
    cell = (np.clip(np.floor(np.stack([r.x, r.y, r.z], 1) * n), 0, n - 1).astype(np.int64)
            @ np.array([1, n, n * n]))
    counts = np.bincount(cell, minlength=n ** 3)
    assert counts[counts > 0].min() == lo and counts.max() == hi
    assert r.added == (lo - 1) * int(a.fluid_mask.sum())
    assert r.removed == (27 - hi) * int(b.fluid_mask.sum())


def test_cfl_number():
    f = facts()
    n = 32
    sc = S.box(n, (0.3, 0.3, 0.3), (0.6, 0.6, 0.6), velocity=(0.0, 0.0, 50.0))
    p = O.Params(n=(n, n, n), dx=1.0 / n, cfl=float(f["cfl_alpha"]))
    assert O.step(p, *sc.arrays(), fields=False).dt == f["cfl_alpha"] * (1.0 / n) / 50.0


def test_marching_cubes_configurations():
    """One cube, every classification of its corners: exactly the two uniform ones
    add no triangles."""
    f = facts()
    empty = 0
    for case in range(f["mc_configurations"]):
        phi = np.ones((2, 2, 2))
        for q in range(8):
            if (case >> q) & 1:
                phi[q >> 2, (q >> 1) & 1, q & 1] = -1.0
        m = O.marching_cubes(phi, (0.0, 0.0, 0.0), 1.0)
        empty += len(m.triangles) == 0
    assert 1 << 8 == f["mc_configurations"]
    assert empty == f["mc_trivial_configurations"]
