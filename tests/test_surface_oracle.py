"""Pins of the surface-reconstruction oracle (Sec. 3.3): the scalar field of Sec.
3.3.1 against closed forms, symmetry and brute force, and the marching cubes of Sec.
3.3.2 against exact planar cases, closedness / orientation of the mesh for every cube
case and for random fields, and the volume and topology of a sphere."""
import itertools
from collections import Counter, deque

import numpy as np
import pytest

import oracle as O
from paper_2404_01931_gb300 import scenes as S


# ------------------------------------------------------------------ scalar field

def test_blobby_kernel_values():
    assert O.blobby_kernel(0.0) == 1.0
    assert O.blobby_kernel(0.5) == 0.421875          # (3/4)^3
    assert O.blobby_kernel(1.0) == 0.0
    assert O.blobby_kernel(1.5) == 0.0
    assert O.blobby_kernel(-0.5) == 0.421875


def _corners(n, origin, h):
    g = [origin[a] + h * np.arange(n[a] + 1) for a in range(3)]
    Z, Y, X = np.meshgrid(g[2], g[1], g[0], indexing="ij")
    return X, Y, Z


def test_single_particle_is_a_sphere():
    n, o, h, r, R = (8, 7, 6), (0.0, 0.1, -0.2), 0.1, 0.05, 0.25
    p = np.array([0.33, 0.41, 0.07])
    phi = O.sdf([p[0]], [p[1]], [p[2]], n, o, h, r, R)
    X, Y, Z = _corners(n, o, h)
    d = np.sqrt((X - p[0]) ** 2 + (Y - p[1]) ** 2 + (Z - p[2]) ** 2)
    want = np.where(d < R, d - r, R - r)
    assert np.abs(phi - want).max() < 1e-14
    assert (d < R).sum() > 20


def test_symmetric_pair_centres_on_the_corner():
    # particles at x +- 0.07 around corner (3, 2, 2): the weighted mean is the corner
    n, o, h, r, R = (6, 4, 4), (0.0, 0.0, 0.0), 0.1, 0.04, 0.2
    c = np.array([0.3, 0.2, 0.2])
    phi = O.sdf([c[0] - 0.07, c[0] + 0.07], [c[1]] * 2, [c[2]] * 2, n, o, h, r, R)
    assert phi[2, 2, 3] == pytest.approx(-r, abs=1e-15)
    # a corner off the pair's axis: the mean is still the midpoint
    assert phi[2, 3, 3] == pytest.approx(0.1 - r, abs=1e-14)


def _brute_sdf(x, y, z, n, o, h, r, R):
    X, Y, Z = _corners(n, o, h)
    out = np.empty(X.shape)
    for idx in np.ndindex(X.shape):
        d = np.stack([x - X[idx], y - Y[idx], z - Z[idx]])
        dist = np.sqrt((d ** 2).sum(0))
        k = np.array([O.blobby_kernel(s) for s in dist / R])
        if k.sum() > 0:
            out[idx] = np.linalg.norm((k * d).sum(1)) / k.sum() - r
        else:
            out[idx] = R - r
    return out


def test_binned_field_equals_brute_force():
    rng = np.random.default_rng(3)
    x, y, z = rng.uniform(-0.1, 0.9, (3, 150))
    n, o, h, r, R = (7, 6, 5), (0.05, 0.0, 0.1), 0.12, 0.03, 0.21
    assert np.abs(O.sdf(x, y, z, n, o, h, r, R) - _brute_sdf(x, y, z, n, o, h, r, R)).max() < 1e-13


def test_field_covariance():
    sc = S.water_drop(12)
    x, y, z = (a.astype(np.float64) for a in (sc.x, sc.y, sc.z))
    n, o, h, r, R = (12, 12, 12), (0.0, 0.0, 0.0), 1 / 12, 0.5 / 12, 2 / 12
    phi = O.sdf(x, y, z, n, o, h, r, R)
    # translation of particles and grid together
    d = (0.013, -0.021, 0.37)
    phi_t = O.sdf(x + d[0], y + d[1], z + d[2], n, tuple(o[a] + d[a] for a in range(3)), h, r, R)
    assert np.abs(phi_t - phi).max() < 1e-12
    # exchange of the x and z axes
    phi_s = O.sdf(z, y, x, n, o, h, r, R)
    assert np.abs(phi_s - phi.transpose(2, 1, 0)).max() < 1e-12
    # uniform scaling of every length
    s = 2.5
    phi_k = O.sdf(s * x, s * y, s * z, n, o, s * h, s * r, s * R)
    assert np.abs(phi_k - s * phi).max() < 1e-12
    assert phi.min() < 0 < phi.max()


def test_symmetric_lattice_interior_is_minus_r():
    # particles on a lattice of spacing h/2 offset by h/4: point-symmetric about every
    # corner, so deep inside the weighted mean is the corner itself
    h = 0.1
    g = (np.arange(24) + 0.5) * h / 2
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    phi = O.sdf(X.ravel(), Y.ravel(), Z.ravel(), (12, 12, 12), (0.0, 0.0, 0.0), h, 0.05, 0.2)
    assert np.abs(phi[3:-3, 3:-3, 3:-3] + 0.05).max() < 1e-13
    assert phi[0, 0, 0] > phi[6, 6, 6]


# ------------------------------------------------------------------ marching cubes

def _edges(tri):
    return Counter((int(a), int(b)) for t in tri for a, b in ((t[0], t[1]), (t[1], t[2]), (t[2], t[0])))


def _closed_and_oriented(tri):
    e = _edges(tri)
    return all(c == 1 and e.get((b, a), 0) == 1 for (a, b), c in e.items())


def _euler(m):
    und = {tuple(sorted(k)) for k in _edges(m.triangles)}
    return len(m.vertices) - len(und) + len(m.triangles)


def _signed_volume(m):
    p = m.vertices[m.triangles]
    return float(np.einsum("ij,ij->i", p[:, 0], np.cross(p[:, 1], p[:, 2])).sum() / 6.0)


def test_plane_is_reproduced_exactly():
    n, h = (9, 9, 9), 1 / 9
    X, Y, Z = _corners(n, (0, 0, 0), h)
    a = np.array([1.0, 1.0, 0.0]) / np.sqrt(2)
    c = 1.03                                    # the plane x + y = c misses every corner
    phi = (X * a[0] + Y * a[1] + Z * a[2]) - c / np.sqrt(2)
    m = O.marching_cubes(phi, (0, 0, 0), h)
    assert len(m.triangles) > 0
    assert np.abs(m.vertices @ a - c / np.sqrt(2)).max() < 1e-14
    assert np.abs(m.normals - a).max() < 1e-12
    p = m.vertices[m.triangles]
    cr = np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0])
    area = 0.5 * np.linalg.norm(cr, axis=1)
    assert (cr @ a > 0).all()
    # inside the unit cube the plane is a rectangle of height 1 and width sqrt(2) (2 - c)
    assert area.sum() == pytest.approx(np.sqrt(2.0) * (2.0 - c), rel=1e-12)


def _case_field(case):
    phi = np.ones((4, 4, 4))
    for q in range(8):
        if (case >> q) & 1:
            phi[1 + (q >> 2), 1 + ((q >> 1) & 1), 1 + (q & 1)] = -1.0
    return phi


def _components(case):
    inside = [q for q in range(8) if (case >> q) & 1]
    seen, comps = set(), 0
    for s in inside:
        if s in seen:
            continue
        comps += 1
        dq = deque([s])
        seen.add(s)
        while dq:
            q = dq.popleft()
            for b in range(3):
                t = q ^ (1 << b)
                if t in inside and t not in seen:
                    seen.add(t)
                    dq.append(t)
    return comps


@pytest.mark.parametrize("case", range(256))
def test_every_cube_case_gives_closed_spheres(case):
    """Every inside/outside pattern of one cube (its neighbours all outside): the mesh
    is closed and consistently wound outward, with one sphere per 6-connected group
    of inside corners (Euler characteristic 2 per group)."""
    phi = _case_field(case)
    m = O.marching_cubes(phi, (0.0, 0.0, 0.0), 1.0)
    comps = _components(case)
    if comps == 0:
        assert len(m.triangles) == 0 and len(m.vertices) == 0
        return
    assert _closed_and_oriented(m.triangles)
    assert _euler(m) == 2 * comps
    assert _signed_volume(m) > 0
    # every crossing edge carries one vertex, and all of them are used
    assert len(np.unique(m.triangles)) == len(m.vertices)
    assert np.all(np.abs(np.linalg.norm(m.normals, axis=1) - 1.0) < 1e-12)


@pytest.mark.parametrize("seed", range(6))
def test_random_fields_give_closed_oriented_meshes(seed):
    rng = np.random.default_rng(seed)
    phi = rng.normal(size=(10, 9, 11)) + 0.2 * seed
    phi[0], phi[-1], phi[:, 0], phi[:, -1], phi[:, :, 0], phi[:, :, -1] = (1.0,) * 6
    m = O.marching_cubes(phi, (0.0, 0.0, 0.0), 1.0)
    assert len(m.triangles) > 50
    assert _closed_and_oriented(m.triangles)
    t = m.triangles
    assert (t[:, 0] != t[:, 1]).all() and (t[:, 1] != t[:, 2]).all() and (t[:, 0] != t[:, 2]).all()
    # the vertex of edge (corner, axis) lies on that edge between the sign change
    c, a = m.vertex_edge // 3, m.vertex_edge % 3
    ijk = np.stack([c % 11, (c // 11) % 9, c // 99], 1).astype(float)
    off = m.vertices - ijk
    for d in range(3):
        on = a == d
        assert ((off[on, d] >= 0) & (off[on, d] <= 1)).all()
        assert np.abs(off[~on, d]).max() == 0.0


def test_sphere_volume_and_topology():
    n, h, rho = 24, 1 / 24, 0.3
    X, Y, Z = _corners((n, n, n), (0, 0, 0), h)
    c = (0.5, 0.48, 0.51)
    phi = np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2) - rho
    m = O.marching_cubes(phi, (0, 0, 0), h)
    assert _closed_and_oriented(m.triangles)
    assert _euler(m) == 2
    v = _signed_volume(m)
    assert v == pytest.approx(4 / 3 * np.pi * rho ** 3, rel=0.02)
    r = np.linalg.norm(m.vertices - np.array(c), axis=1)
    assert np.abs(r - rho).max() < 0.05 * h
    # outward normals
    assert (np.einsum("ij,ij->i", m.normals, m.vertices - np.array(c)) > 0).all()


# ------------------------------------------------------------------ library table

def test_library_case_table_matches_the_oracle():
    """Host logic of the CUDA library: its generated case table lists, for every
    corner pattern, exactly the triangles (as local edges, in order) that the oracle
    finds by polygonising that cube directly."""
    from paper_2404_01931_gb300 import flip as F
    ntri, tri = F.surface_case_table()
    for case in range(256):
        phi = np.array([[[-1.0 if (case >> (i + 2 * j + 4 * k)) & 1 else 1.0 for i in range(2)]
                         for j in range(2)] for k in range(2)])
        m = O.marching_cubes(phi, (0.0, 0.0, 0.0), 1.0)
        corner, axis = m.vertex_edge // 3, m.vertex_edge % 3
        bits = np.stack([corner % 2, (corner // 2) % 2, corner // 4], 1)
        lo = np.where(axis == 0, 1, 0)
        hi = np.where(axis == 2, 1, 2)
        local = 4 * axis + bits[np.arange(len(axis)), lo] + 2 * bits[np.arange(len(axis)), hi]
        want = local[m.triangles] if len(m.triangles) else np.zeros((0, 3), int)
        assert ntri[case] == len(want), case
        assert np.array_equal(tri[case, :ntri[case]], want), case
