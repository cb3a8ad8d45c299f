"""Seeded scene generator: sizes of the measured workloads, determinism, jitter layout."""
import numpy as np

from paper_2404_01931_gb300 import scenes as S


def test_splitmix64_reference_values():
    # SplitMix64 stream from state 0 (Steele, Lea, Flood 2014): first outputs
    got = S.splitmix64(np.arange(3), 0)
    assert [int(v) for v in got] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_dam_break_32_sizes():
    s = S.dam_break(32)
    assert s.n_particles == 32768 and s.fluid_mask.sum() == 4096
    assert s.x.dtype == np.float32 and s.x.max() < 0.25 and s.y.max() < 0.5


def test_pool_drop_cell_count():
    # 77 pool layers of 256^2 plus the sphere cells above them
    _, cy, _ = S.cell_centres((256, 256, 256), 1 / 256)
    assert (cy < 0.3).sum() == 5046272


def test_jitter_one_particle_per_subcell():
    s = S.dam_break(16, 0.25, 0.25, seed=3)
    dx = 1 / 16
    g = np.stack([s.x, s.y, s.z], 1).astype(np.float64) / dx * 2
    sub = np.floor(g).astype(np.int64)
    key = sub[:, 0] + 32 * (sub[:, 1] + 32 * sub[:, 2])
    assert np.unique(key).size == s.n_particles
    assert s.fluid_mask.sum() * 8 == s.n_particles


def test_deterministic_and_seed_dependent():
    a = S.dam_break(16, seed=1)
    b = S.dam_break(16, seed=1)
    c = S.dam_break(16, seed=2)
    assert np.array_equal(a.x, b.x) and not np.array_equal(a.x, c.x)


def test_batch_scenes_uneven():
    sc = S.batch_scenes(8, seed=0)
    edges = {s.n[0] for s in sc}
    assert len(sc) == 8 and edges <= {32, 48, 64, 80, 96} and len(edges) > 1
