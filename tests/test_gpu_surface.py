"""Surface reconstruction (Sec. 3.3) on the CUDA path against the FP64 oracle,
through the C ABI (include/flip_surface.h).

Marching cubes from the same float32 field: the mesh topology is integer work and
must be identical (vertex edges, triangle lists, counts); vertex positions agree to
FP32 rounding of origin + h (i + t); normals agree where the triangles around a
vertex are well shaped (the inverse-area weights of Sec. 3.3.2 amplify the rounding
of near-degenerate triangles).  The scalar field of Sec. 3.3.1 from the same float32
particles agrees to FP32 rounding of the kernel sums."""
from collections import Counter

import numpy as np
import pytest

import oracle as O
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


def _sp(n, h, origin=(0.0, 0.0, 0.0), r=None, R=None, iso=0.0):
    sp = F.FlipSurfaceParams()
    for a in range(3):
        sp.n[a] = n[a]
        sp.origin[a] = origin[a]
    sp.h = h
    sp.radius = 0.5 * h if r is None else r
    sp.search_radius = 2.0 * h if R is None else R
    sp.iso = iso
    return sp


def _gpu_mesh(sp, phi):
    with F.Surface(sp) as s:
        s.set_field(phi)
        nv, nt = s.mesh()
        out = {k: s.read(w) for k, w in (("v", F.SURF_VERTICES), ("n", F.SURF_NORMALS),
                                         ("t", F.SURF_TRIANGLES), ("e", F.SURF_VERTEX_EDGE))}
    return nv, nt, out


def _areas(vert, tri):
    p = vert[tri]
    return 0.5 * np.linalg.norm(np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), axis=1)


def _compare_mesh(sp, phi, label=""):
    n = tuple(sp.n)
    origin = tuple(sp.origin)
    ref = O.marching_cubes(phi.astype(np.float64), origin, sp.h, float(np.float32(sp.iso)))
    nv, nt, got = _gpu_mesh(sp, phi)
    assert (nv, nt) == (len(ref.vertices), len(ref.triangles)), label
    assert np.array_equal(got["e"], ref.vertex_edge), label
    assert np.array_equal(got["t"], ref.triangles), label
    scale = max(abs(o) for o in origin) + sp.h * max(n)
    dv = np.abs(got["v"].astype(np.float64) - ref.vertices).max() if nv else 0.0
    assert dv <= 4e-7 * scale + 1e-6 * sp.h, (label, dv)
    if nt:
        # Normals where every triangle at the vertex has area >= 1e-2 h^2.  The GPU
        # takes edge vectors from float32 vertices of magnitude ~scale, so an edge of
        # length L carries a relative error ~6e-8 scale / L; for such triangles
        # (L >~ 0.14 h, scale/h <= 64 here) that is <~ 3e-5 in each unit normal and
        # <~ 6e-5 in each inverse-area weight, and the weighted sum of normals that
        # differ by up to ~2 moves by <~ 2e-4; smaller triangles grow as 1/area.
        small = _areas(ref.vertices, ref.triangles) < 1e-2 * sp.h ** 2
        bad = np.zeros(nv, bool)
        bad[ref.triangles[small].ravel()] = True
        good = ~bad
        dn = np.abs(got["n"][good].astype(np.float64) - ref.normals[good]).max()
        assert dn <= 5e-4, (label, dn)
        ln = np.linalg.norm(got["n"].astype(np.float64), axis=1)
        assert np.all((ln == 0) | (np.abs(ln - 1) < 1e-5)), label
    return nv, nt


def test_mesh_of_a_noisy_sphere():
    n, h = (40, 40, 40), 1 / 40
    phi = S.corner_field_sphere(n, h, (0.5, 0.48, 0.53), 0.31, noise=0.3 * h, seed=1)
    nv, nt = _compare_mesh(_sp(n, h), phi, "sphere")
    assert nt > 5000


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_mesh_of_random_fields_ragged_grid(seed):
    n = (13, 7, 21)
    phi = S.corner_field_random(n, seed, bias=0.1 * seed)
    _compare_mesh(_sp(n, 0.37, origin=(-1.5, 0.25, 3.0)), phi, f"random {seed}")


def test_mesh_of_open_random_field_and_iso():
    """Boundary corners not forced outside (open surfaces), a nonzero isovalue, and
    corners lying exactly on it."""
    n = (24, 17, 9)
    phi = S.corner_field_random(n, 5, closed=False)
    phi[::3, ::2, ::4] = np.float32(0.25)
    _compare_mesh(_sp(n, 0.1, iso=0.25), phi, "open iso")


@pytest.mark.parametrize("value", [1.0, -1.0])
def test_mesh_without_crossings_is_empty(value):
    n = (5, 6, 7)
    nv, nt, _ = _gpu_mesh(_sp(n, 0.1), np.full((8, 7, 6), value, np.float32))
    assert (nv, nt) == (0, 0)


def test_every_cube_case_on_one_cube():
    sp = _sp((1, 1, 1), 1.0)
    ntri, _ = F.surface_case_table()
    with F.Surface(sp) as s:
        for case in range(256):
            phi = np.array([[[-1.0 if (case >> (i + 2 * j + 4 * k)) & 1 else 1.0 for i in range(2)]
                             for j in range(2)] for k in range(2)], np.float32)
            s.set_field(phi)
            nv, nt = s.mesh()
            ref = O.marching_cubes(phi.astype(np.float64), (0, 0, 0), 1.0)
            assert nt == ntri[case] == len(ref.triangles)
            assert np.array_equal(s.read(F.SURF_TRIANGLES), ref.triangles), case


def _sdf_case(sc, sp, label):
    fp = matched(sc.n)[1]
    with F.Simulation(fp, *sc.arrays()) as sim, F.Surface(sp) as s:
        s.sdf(sim)
        phi = s.read(F.SURF_FIELD).astype(np.float64)
    ref = O.sdf(sc.x, sc.y, sc.z, tuple(sp.n), tuple(sp.origin), sp.h, sp.radius,
                sp.search_radius)
    err = np.abs(phi - ref)
    # FP32 kernel sums: relative rounding ~1e-6 of the lengths involved (R)
    assert err.max() <= 2e-5 * sp.search_radius, (label, err.max() / sp.search_radius)
    assert (ref < 0).sum() > 100 and (ref > 0).sum() > 100
    return phi, ref


def test_sdf_matches_the_oracle_default_grid():
    sc = S.water_drop(32)
    fp = matched(32)[1]
    sp = F.surface_default_params(fp)
    assert tuple(sp.n) == (32, 32, 32) and sp.h == fp.dx
    _sdf_case(sc, sp, "water drop 32")


def test_sdf_matches_the_oracle_finer_offset_grid():
    sc = S.random_velocities(S.double_dam_break(24), 0.2, 1)
    sp = _sp((50, 41, 47), 0.021, origin=(-0.013, 0.004, 0.011), r=0.6 / 24, R=1.7 / 24)
    _sdf_case(sc, sp, "double dam break, finer grid")


def test_sdf_to_mesh_of_a_drop_is_closed():
    sc = S.water_drop(48)
    fp = matched(48)[1]
    sp = F.surface_default_params(fp)
    with F.Simulation(fp, *sc.arrays()) as sim, F.Surface(sp) as s:
        s.sdf(sim)
        nv, nt = s.mesh()
        tri = s.read(F.SURF_TRIANGLES)
        vert = s.read(F.SURF_VERTICES).astype(np.float64)
    e = Counter((int(a), int(b)) for t in tri for a, b in ((t[0], t[1]), (t[1], t[2]), (t[2], t[0])))
    assert all(c == 1 and e.get((b, a), 0) == 1 for (a, b), c in e.items())
    p = vert[tri]
    vol = np.einsum("ij,ij->i", p[:, 0], np.cross(p[:, 1], p[:, 2])).sum() / 6
    assert vol == pytest.approx(4 / 3 * np.pi * 0.2 ** 3, rel=0.15)


def test_surface_argument_errors():
    with pytest.raises(F.FlipError):
        F.Surface(_sp((0, 4, 4), 0.1))
    with pytest.raises(F.FlipError):
        F.Surface(_sp((4, 4, 4), 0.1, r=0.3, R=0.2))
    with F.Surface(_sp((4, 4, 4), 0.1)) as s:
        buf = np.zeros(3, np.float32)
        rc = F.lib().flip_surface_read(s.h, F.SURF_FIELD, buf.ctypes.data, buf.nbytes, 0)
        assert rc == F.FLIP_E_SIZE


def test_sdf_follows_a_reseeding_handle():
    """The scalar field reads the handle's current particle count, which reseeding
    changes from step to step; the drop's mesh stays closed."""
    sc = S.water_drop(40)
    fp = matched(40)[1]
    fp.ppc_min, fp.ppc_max = 3, 12
    with F.Simulation(fp, *sc.arrays()) as sim, F.Surface(F.surface_default_params(fp)) as s:
        for _ in range(3):
            rc, st = sim.step(4, stats=True)
            assert rc == F.FLIP_OK
            s.sdf(sim)
            nv, nt = s.mesh()
            tri = s.read(F.SURF_TRIANGLES)
            e = Counter((int(a), int(b)) for t in tri for a, b in ((t[0], t[1]), (t[1], t[2]), (t[2], t[0])))
            assert nt > 100 and all(c == 1 and e.get((b, a), 0) == 1 for (a, b), c in e.items())
        assert st.n_particles == len(sim.read(F.PX))
