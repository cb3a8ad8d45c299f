"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test ties one part of the oracle to something other than itself:

  part (paper passage)                 pin
  -----------------------------------  ------------------------------------------------
  hat function (Eq. 4b)                exact values of the piecewise-linear definition
  weights (Eq. 4a, near-wall reading)  partition of unity over *all* nodes; linear
                                       fields interpolated exactly at the clamped point
  binning (Sec. 3.1.5)                 numpy stable argsort of floor(x/dx)
  P2G gather (Sec. 3.1.6)              brute force over every particle and every face;
                                       a uniform field survives P2G -> G2P exactly
  divergence (Eq. 6)                   linear field: div = a + b + c everywhere
  Laplacian (Sec. 3.1.7)               symmetric, Cholesky-positive, row sums; closed-form
                                       spectrum of a fluid layer (Neumann/Dirichlet paths)
  PCG (Sec. 3.1.7)                     dense LAPACK solve on random 4^3-8^3 masks
  projection (Eq. 5)                   post-projection divergence = 0 (numpy div);
                                       projecting twice gives p = 0
  gravity + G2P + advection            ballistic closed form v = v0 + n g dt,
  (Eq. 1, Secs. 3.1.3, 3.1.8)          x = x0 + n dt v0 + g dt^2 n(n+1)/2
  FLIP/PIC blend (Sec. 2.1.4, 3.1.8)   shifted grid field: v = r(v+c) + (1-r)(U0+c)
  full step                            hydrostatic column p_j = rho g (H - j) dx, at rest
"""
import numpy as np
import pytest

from paper_2404_01931_gb300 import scenes as S

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _params(O, n, **kw):
    n = tuple(n) if not np.isscalar(n) else (n, n, n)
    kw.setdefault("dx", 1.0 / max(n))
    return O.Params(n=n, **kw)


# ---------------------------------------------------------------- Eq. 4 weights

def test_hat_values(oracle_mod):
    O = oracle_mod
    for r, h in [(0.0, 1.0), (1.0, 0.0), (-1.0, 0.0), (0.5, 0.5), (-0.25, 0.75),
                 (1.5, 0.0), (-3.0, 0.0), (0.999, 0.001)]:
        assert O.hat(r) == pytest.approx(h, abs=1e-15)


def test_partition_of_unity_all_nodes(oracle_mod):
    """Sum of Eq. 4 weights over every node of the grid is 1 (points near walls too)."""
    O = oracle_mod
    n = (5, 4, 6)
    P = _params(O, n, dx=0.1)
    rng = np.random.default_rng(1)
    pts = rng.uniform(0, 1, (40, 3)) * np.array(n) * 0.1
    pts[:6] = [[0.0, 0.0, 0.0], [0.5 - 1e-12, 0.4 - 1e-12, 0.6 - 1e-12], [0.01, 0.39, 0.3],
               [0.049, 0.051, 0.599], [0.25, 0.2, 0.0], [0.5, 0.05, 0.05]]
    for comp in range(3):
        shp = O.face_shape(n, comp)
        for x, y, z in pts:
            tot = 0.0
            for c in range(shp[0]):
                for b in range(shp[1]):
                    for a in range(shp[2]):
                        w = O.weight(P, comp, (a, b, c), x, y, z)
                        assert w >= 0.0
                        tot += w
            assert tot == pytest.approx(1.0, abs=1e-14)


def test_interp_reproduces_linear_fields(oracle_mod):
    """Trilinear interpolation of a linear function sampled at the face nodes returns
    the function at the particle (interior) or at the clamped sample point (near walls)."""
    O = oracle_mod
    n = (6, 5, 7)
    dx = 0.125
    P = _params(O, n, dx=dx)
    rng = np.random.default_rng(2)
    coef = rng.normal(size=4)
    pts = rng.uniform(0, 1, (60, 3)) * np.array(n) * dx
    for comp in range(3):
        shp = O.face_shape(n, comp)
        off = np.array([0.5, 0.5, 0.5])
        off[comp] = 0.0
        c_, b_, a_ = np.meshgrid(*[np.arange(s) for s in shp], indexing="ij")
        fld = coef[0] + coef[1] * (a_ + off[0]) * dx + coef[2] * (b_ + off[1]) * dx \
            + coef[3] * (c_ + off[2]) * dx
        got = O.interp(P, comp, fld, pts[:, 0], pts[:, 1], pts[:, 2])
        # clamped sample point, axis by axis: node range is [off, dim-1+off] * dx
        lo = off * dx
        hi = (np.array([shp[2], shp[1], shp[0]]) - 1 + off) * dx
        q = np.clip(pts, lo, hi)
        want = coef[0] + q @ coef[1:]
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)


# ---------------------------------------------------------------- binning

def test_binning_matches_stable_argsort(oracle_mod):
    O = oracle_mod
    n = (7, 5, 6)
    P = _params(O, n, dx=0.1)
    rng = np.random.default_rng(3)
    pts = rng.uniform(-0.05, 0.75, (500, 3))
    pts[:5] = [[0.1, 0.2, 0.3], [0.0, 0.0, 0.0], [0.7, 0.5, 0.6], [0.69999, 0.49999, 0.59999],
               [-0.01, 0.51, 0.3]]
    start, order = O.bin_particles(P, pts[:, 0], pts[:, 1], pts[:, 2])
    # the documented binning rule: floor(x * (1/dx)) per axis, clamped to the grid
    ijk = np.clip(np.floor(pts * (1.0 / 0.1)).astype(np.int64), 0, np.array(n) - 1)
    cid = ijk[:, 0] + n[0] * (ijk[:, 1] + n[1] * ijk[:, 2])
    np.testing.assert_array_equal(order, np.argsort(cid, kind="stable"))
    np.testing.assert_array_equal(np.diff(start), np.bincount(cid, minlength=int(np.prod(n))))


# ---------------------------------------------------------------- P2G (Sec. 3.1.6)

def _brute_p2g(n, dx, comp, pts, vel):
    """Every particle against every face node, Eq. 4 on the clamped coordinate."""
    shp = [n[0] + (comp == 0), n[1] + (comp == 1), n[2] + (comp == 2)]
    off = np.array([0.5, 0.5, 0.5])
    off[comp] = 0.0
    g = np.clip(pts / dx - off, 0, np.array(shp) - 1)  # (np, 3)
    num = np.zeros((shp[2], shp[1], shp[0]))
    den = np.zeros_like(num)
    for c in range(shp[2]):
        for b in range(shp[1]):
            for a in range(shp[0]):
                w = np.prod(np.maximum(0.0, 1.0 - np.abs(g - np.array([a, b, c]))), axis=1)
                num[c, b, a] = np.sum(w * vel)
                den[c, b, a] = np.sum(w)
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.where(den > 0, num / den, 0.0), den


@pytest.mark.parametrize("comp", [0, 1, 2])
def test_p2g_gather_equals_brute_force(oracle_mod, comp):
    O = oracle_mod
    n = (5, 6, 4)
    dx = 0.1
    P = _params(O, n, dx=dx)
    rng = np.random.default_rng(10 + comp)
    pts = rng.uniform(0, 1, (300, 3)) * np.array(n) * dx
    pts[:4] = [[0.0, 0.0, 0.0], [0.5 - 1e-9, 0.6 - 1e-9, 0.4 - 1e-9], [0.02, 0.3, 0.39],
               [0.25, 0.05, 0.2]]
    # leave a hole so some faces stay empty
    keep = ~((pts[:, 0] > 0.3) & (pts[:, 1] > 0.35))
    pts = pts[keep]
    vel = rng.normal(size=pts.shape[0])
    got, ws = O.p2g(P, comp, pts[:, 0], pts[:, 1], pts[:, 2], vel)
    want, den = _brute_p2g(n, dx, comp, pts, vel)
    np.testing.assert_allclose(ws, den, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-13)
    assert (den == 0).any() and (den > 0).any()


def test_uniform_field_survives_p2g_g2p(oracle_mod):
    """All particles share one velocity: P2G gives it on every reached face, and
    G2P with the unchanged field returns it exactly for any FLIP ratio."""
    O = oracle_mod
    n = (8, 8, 8)
    rng = np.random.default_rng(4)
    sc = S.box(n, (0.0, 0.0, 0.0), (0.6, 0.8, 1.0), seed=3)
    vel0 = rng.normal(size=3)
    for ratio in (0.0, 0.95, 1.0):
        P = _params(O, n, flip_ratio=ratio, gravity=(0.0, 0.0, 0.0))
        uo = []
        for d in range(3):
            g, ws = O.p2g(P, d, sc.x, sc.y, sc.z, np.full(sc.n_particles, vel0[d]))
            reached = ws > 0
            np.testing.assert_allclose(g[reached], vel0[d], rtol=1e-14, atol=1e-15)
            assert np.all(g[~reached] == 0.0)
            uo.append(g)
        out = O.g2p(P, sc.x, sc.y, sc.z, *[np.full(sc.n_particles, vel0[d]) for d in range(3)],
                    uo, uo)
        for d in range(3):
            np.testing.assert_allclose(out[3 + d], vel0[d], rtol=1e-14, atol=1e-15)


# ---------------------------------------------------------------- Eq. 6 divergence

def test_divergence_of_linear_field(oracle_mod):
    O = oracle_mod
    n = (5, 4, 6)
    dx = 0.2
    P = _params(O, n, dx=dx)
    a, b, c = 1.7, -0.4, 2.3
    flds = []
    for comp, coef in enumerate((a, b, c)):
        shp = O.face_shape(n, comp)
        pos = np.arange(shp[2 - comp]) * dx  # node position along the component's own axis
        f = np.zeros(shp)
        if comp == 0:
            f[:] = coef * pos[None, None, :]
        elif comp == 1:
            f[:] = coef * pos[None, :, None]
        else:
            f[:] = coef * pos[:, None, None]
        flds.append(f + 0.37)
    t = np.ones(O.cell_shape(n), np.uint8)
    t[0, 0, 0] = 0
    bb = O.divergence(P, flds, t)
    want = np.full(O.cell_shape(n), -(a + b + c))
    want[0, 0, 0] = 0.0
    np.testing.assert_allclose(bb, want, rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------- Laplacian (Sec. 3.1.7)

def _dense_A(O, P, t):
    fl = np.flatnonzero(t.ravel())
    A = np.zeros((fl.size, fl.size))
    e = np.zeros(t.size)
    for col, c in enumerate(fl):
        e[:] = 0.0
        e[c] = 1.0
        A[:, col] = O.apply_A(P, t, e.reshape(t.shape)).ravel()[fl]
    return A, fl


@pytest.mark.parametrize("n,seed", [((4, 4, 4), 0), ((6, 5, 4), 1), ((8, 8, 8), 2)])
def test_laplacian_symmetric_pd_rowsums(oracle_mod, n, seed):
    O = oracle_mod
    P = _params(O, n, dt=0.01, rho=2.0)
    t = S.random_mask(n, 0.6, seed).astype(np.uint8)
    A, fl = _dense_A(O, P, t)
    assert np.array_equal(A, A.T)
    np.linalg.cholesky(A)
    s = P.dt / (P.rho * P.dx ** 2)
    nx, ny, nz = n
    for row, c in enumerate(fl):
        i, j, k = c % nx, (c // nx) % ny, c // (nx * ny)
        air = 0
        for di, dj, dk in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
            ii, jj, kk = i + di, j + dj, k + dk
            if 0 <= ii < nx and 0 <= jj < ny and 0 <= kk < nz and not t[kk, jj, ii]:
                air += 1
        assert A[row].sum() == pytest.approx(s * air, abs=1e-9 * s)


@pytest.mark.parametrize("n,H", [((4, 6, 3), 4), ((5, 7, 4), 2), ((3, 9, 5), 8)])
def test_laplacian_spectrum_of_layer(oracle_mod, n, H):
    """Fluid layer j < H over the whole floor: walls on x, z and the floor (Neumann),
    air above (Dirichlet).  A = s (Lx + Ly + Lz) with closed-form path spectra."""
    O = oracle_mod
    P = _params(O, n, dt=0.02, rho=1.5)
    t = np.zeros(O.cell_shape(n), np.uint8)
    t[:, :H, :] = 1
    A, _ = _dense_A(O, P, t)
    s = P.dt / (P.rho * P.dx ** 2)
    nx, _, nz = n
    lx = 2 - 2 * np.cos(np.pi * np.arange(nx) / nx)
    lz = 2 - 2 * np.cos(np.pi * np.arange(nz) / nz)
    ly = 2 - 2 * np.cos(np.pi * (2 * np.arange(H) + 1) / (2 * H + 1))
    want = np.sort((lx[None, None, :] + ly[None, :, None] + lz[:, None, None]).ravel()) * s
    got = np.linalg.eigvalsh(A)
    np.testing.assert_allclose(got, want, rtol=1e-10, atol=1e-10 * s)


@pytest.mark.parametrize("n,seed", [((4, 4, 4), 5), ((6, 7, 5), 6), ((8, 8, 8), 7)])
def test_pcg_matches_dense_solve(oracle_mod, n, seed):
    O = oracle_mod
    P = _params(O, n, dt=1 / 240)
    t = S.random_mask(n, 0.7, seed).astype(np.uint8)
    rng = np.random.default_rng(seed)
    b = rng.normal(size=t.shape) * t
    x, it, rel = O.pcg(P, t, b, tol=1e-13, max_iter=10000)
    assert it > 0 and rel <= 1e-13
    A, fl = _dense_A(O, P, t)
    xd = np.linalg.solve(A, b.ravel()[fl])
    err = np.linalg.norm(x.ravel()[fl] - xd) / np.linalg.norm(xd)
    assert err <= 1e-10
    assert np.all(x.ravel()[np.flatnonzero(t.ravel() == 0)] == 0.0)


def test_pcg_zero_rhs_returns_zero(oracle_mod):
    O = oracle_mod
    P = _params(O, 4)
    t = np.ones(O.cell_shape((4, 4, 4)), np.uint8)
    t[3] = 0
    x, it, rel = O.pcg(P, t, np.zeros(t.shape))
    assert it == 0 and np.all(x == 0)


# ---------------------------------------------------------------- projection (Eq. 5)

def _numpy_div(n, dx, u3, t):
    d = (np.diff(u3[0], axis=2) + np.diff(u3[1], axis=1) + np.diff(u3[2], axis=0)) / dx
    return d * t


def test_projection_removes_divergence_and_is_idempotent(oracle_mod):
    O = oracle_mod
    n = (12, 12, 12)
    sc = S.random_velocities(S.box(n, (0.0, 0.0, 0.0), (0.5, 0.6, 1.0), seed=1), 0.5, 9)
    P = _params(O, n, cg_tol=1e-13, cg_max_iter=5000)
    r = O.step(P, *sc.arrays())
    assert r.status == 0
    d_star = np.linalg.norm(_numpy_div(n, P.dx, r.u_star, r.type))
    d_new = np.linalg.norm(_numpy_div(n, P.dx, r.u_new, r.type))
    assert d_star > 0 and d_new / d_star <= 1e-11
    assert r.rel_divergence == pytest.approx(d_new / d_star, rel=1e-6, abs=1e-14)
    # second projection of the projected field: right-hand side ~ 0, pressure ~ 0
    b2 = O.divergence(P, r.u_new, r.type)
    p2, _, _ = O.pcg(P, r.type, b2, tol=1e-13, max_iter=5000)
    assert np.abs(p2).max() <= 1e-9 * np.abs(r.pressure).max()
    # wall faces are zero; faces between two air cells keep u*
    assert np.all(r.u_new[0][:, :, 0] == 0) and np.all(r.u_new[0][:, :, -1] == 0)
    assert np.all(r.u_new[1][:, 0, :] == 0) and np.all(r.u_new[1][:, -1, :] == 0)
    assert np.all(r.u_new[2][0] == 0) and np.all(r.u_new[2][-1] == 0)
    t = r.type.astype(bool)
    airair = ~t[:, 1:, :] & ~t[:, :-1, :]
    np.testing.assert_array_equal(r.u_new[1][:, 1:-1, :][airair], r.u_star[1][:, 1:-1, :][airair])


# ---------------------------------------------------------------- full-step closed forms

def test_ballistic_blob(oracle_mod):
    """A blob away from the walls, all particles with one velocity: div u* = 0, p = 0,
    and the FLIP step is free fall: v_n = v0 + n g dt, x_n = x0 + n dt v0 + g dt^2 n(n+1)/2."""
    O = oracle_mod
    n = (16, 16, 16)
    v0 = np.array([0.3, 0.5, -0.2])
    sc = S.box(n, (0.3, 0.4, 0.3), (0.6, 0.7, 0.55), seed=2, velocity=v0)
    g = np.array([0.0, -9.81, 0.0])
    dt = 1 / 240
    P = _params(O, n, dt=dt, gravity=tuple(g), flip_ratio=0.95)
    st = [a.astype(np.float64) for a in sc.arrays()]
    x0 = np.stack(st[:3], 1)
    steps = 5
    for _ in range(steps):
        r = O.step(P, *st)
        # div u* is rounding noise only (normalised averages of equal values)
        assert r.status == 0 and np.abs(r.rhs).max() <= 1e-12
        assert np.abs(r.pressure).max() <= 1e-14
        st = [r.x, r.y, r.z, r.u, r.v, r.w]
    vel = np.stack(st[3:], 1)
    pos = np.stack(st[:3], 1)
    np.testing.assert_allclose(vel, np.broadcast_to(v0 + steps * g * dt, vel.shape), atol=1e-12)
    want = x0 + steps * dt * v0 + g * dt * dt * steps * (steps + 1) / 2
    np.testing.assert_allclose(pos, want, atol=1e-12)


def test_flip_pic_blend_closed_form(oracle_mod):
    O = oracle_mod
    n = (6, 6, 6)
    sc = S.box(n, (0.1, 0.1, 0.1), (0.9, 0.9, 0.9), seed=5)
    rng = np.random.default_rng(6)
    U0 = rng.normal(size=3)
    c = rng.normal(size=3)
    vp = [rng.normal(size=sc.n_particles) for _ in range(3)]
    for ratio in (0.0, 0.3, 0.95, 1.0):
        for src in (0, 1):
            P = _params(O, n, flip_ratio=ratio, advect_source=src, dt=0.01, skin=0.0)
            uo = [np.full(O.face_shape(n, d), U0[d]) for d in range(3)]
            un = [uo[d] + c[d] for d in range(3)]
            out = O.g2p(P, sc.x, sc.y, sc.z, *vp, uo, un)
            for d in range(3):
                want_v = ratio * (vp[d] + c[d]) + (1 - ratio) * (U0[d] + c[d])
                np.testing.assert_allclose(out[3 + d], want_v, atol=1e-14)
                adv = want_v if src == 0 else U0[d] + c[d]
                xd = np.array((sc.x, sc.y, sc.z)[d], np.float64)
                np.testing.assert_allclose(out[d], np.clip(xd + 0.01 * adv, 0.0, 1.0), atol=1e-14)


def test_wall_clamp(oracle_mod):
    O = oracle_mod
    n = (4, 4, 4)
    P = _params(O, n, dt=1.0, flip_ratio=1.0, skin=1e-3 / 4)
    z = [np.zeros(O.face_shape(n, d)) for d in range(3)]
    out = O.g2p(P, [0.1, 0.9], [0.5, 0.5], [0.5, 0.02], [-5.0, 5.0], [0.0, 0.0], [0.0, -1.0], z, z)
    assert out[0][0] == P.c().skin and out[0][1] == 1.0 - P.c().skin
    assert out[2][1] == P.c().skin and out[1][0] == 0.5


@pytest.mark.parametrize("H", [16, 7])
def test_hydrostatic_column(oracle_mod, H):
    """Full-width layer of H cells at rest: p_j = rho g (H - j) dx exactly (p is linear in
    y, so the discrete Laplacian is exact), u_new = 0 on interior faces, particles stay."""
    O = oracle_mod
    n = (32, 32, 32) if H == 16 else (12, 20, 9)
    sc = S.layer(n, H, seed=4)
    P = _params(O, n, cg_tol=1e-13, cg_max_iter=20000, rho=1.0)
    g = 9.81
    st = [a.astype(np.float64) for a in sc.arrays()]
    x0 = np.stack(st[:3], 1)
    steps = 10 if H == 16 else 3
    for s in range(steps):
        r = O.step(P, *st)
        assert r.status == 0
        st = [r.x, r.y, r.z, r.u, r.v, r.w]
        if s == 0:
            jj = np.arange(n[1])
            want = np.where(jj < H, P.rho * g * (H - jj) * P.dx, 0.0)
            want = np.broadcast_to(want[None, :, None], r.pressure.shape)
            np.testing.assert_allclose(r.pressure, want, rtol=1e-10, atol=1e-12)
            fl = r.type.astype(bool)
            np.testing.assert_allclose(r.u_new[1][:, 1:H + 1, :], 0.0, atol=1e-10 * g * P.dt)
            assert fl[:, :H, :].all() and not fl[:, H:, :].any()
    speed = np.sqrt(st[3] ** 2 + st[4] ** 2 + st[5] ** 2)
    assert speed.max() <= 1e-8 * g * P.dt
    # seeding may place a particle closer to a wall than the skin width; the clamp of
    # Sec. 3.1.3 moves it out on the first step and nothing moves afterwards
    skin = P.c().skin
    x0 = np.clip(x0, skin, np.array(n) * P.dx - skin)
    np.testing.assert_allclose(np.stack(st[:3], 1), x0, atol=1e-6 * P.dx)


def test_singular_closed_box_is_refused(oracle_mod):
    O = oracle_mod
    n = (4, 4, 4)
    sc = S.box(n, (0, 0, 0), (1, 1, 1), seed=1)
    r = O.step(_params(O, n), *sc.arrays())
    assert r.status == 2


def test_dam_break_first_step_sane(oracle_mod):
    """The 32^3 dam break: converges, divergence reduced to the solver tolerance,
    momentum points down and toward the open side."""
    O = oracle_mod
    sc = S.dam_break(32)
    P = _params(O, 32)
    r = O.step(P, *sc.arrays())
    assert r.status == 0 and 0 < r.cg_iterations < 640
    assert r.rel_divergence <= 1.5e-6
    assert r.n_fluid == 4096
    assert r.v.mean() < 0 and r.u.mean() > 0


# ---------------------------------------------------------------- multigrid preconditioner

def test_mg_level_shapes(oracle_mod):
    O = oracle_mod
    assert O.mg_levels(_params(O, 256)) == [(256,) * 3, (128,) * 3, (64,) * 3, (32,) * 3,
                                            (16,) * 3, (8,) * 3, (4,) * 3]
    assert O.mg_levels(_params(O, (20, 13, 17))) == [(20, 13, 17), (10, 7, 9), (5, 4, 5),
                                                     (3, 2, 3)]
    assert O.mg_levels(_params(O, 4)) == [(4, 4, 4)]


def _dense_M(O, P, t, nu, omega):
    fl = np.flatnonzero(t.ravel())
    M = np.zeros((fl.size, fl.size))
    e = np.zeros(t.size)
    for col, c in enumerate(fl):
        e[:] = 0.0
        e[c] = 1.0
        M[:, col] = O.mg_vcycle(P, t, e.reshape(t.shape), nu, omega).ravel()[fl]
    return M, fl


@pytest.mark.parametrize("n,box,nu", [((8, 8, 8), (4, 6, 8), 1), ((16, 16, 16), (8, 12, 16), 2),
                                       ((16, 8, 12), (12, 4, 8), 2)])
def test_mg_vcycle_galerkin_spectrum_in_unit_interval(oracle_mod, n, box, nu):
    """omega = 1 on a fluid box aligned with the coarsest blocks: every coarse cell is
    all fluid or all air, so the rediscretised coarse operator equals the Galerkin one
    (P^T A P = 16 A_c for piecewise-constant P, hence restriction P^T/16), the
    post-smoother reverses the pre-smoother's colour order, and I - M^-1 A is
    A-non-negative: eig(M^-1 A) lies in (0, 1].  A wrong restriction scale, colour
    order or coarse scale pushes eigenvalues out."""
    O = oracle_mod
    P = _params(O, n, dt=1 / 240)
    t = np.zeros(O.cell_shape(n), np.uint8)
    t[:box[2], :box[1], :box[0]] = 1
    assert len(O.mg_levels(P)) >= 2
    M, fl = _dense_M(O, P, t, nu, 1.0)
    assert np.abs(M - M.T).max() <= 1e-12 * np.abs(M).max()
    A, fl2 = _dense_A(O, P, t)
    assert np.array_equal(fl, fl2)
    ev = np.linalg.eigvals(M @ A)
    assert np.abs(ev.imag).max() <= 1e-9
    assert ev.real.min() > 0 and ev.real.max() <= 1 + 1e-9


@pytest.mark.parametrize("n,seed", [((8, 8, 8), 1), ((10, 9, 11), 2), ((6, 12, 5), 3)])
@pytest.mark.parametrize("omega", [1.0, 2.0])
def test_mg_vcycle_random_mask_is_spd(oracle_mod, n, seed, omega):
    """Any mask, any omega > 0: the cycle is symmetric positive definite (symmetrised
    smoother plus a positively scaled SPD coarse term)."""
    O = oracle_mod
    P = _params(O, n, dt=1 / 240)
    t = S.random_mask(n, 0.65, seed).astype(np.uint8)
    M, _ = _dense_M(O, P, t, O.MG_NU, omega)
    assert np.abs(M - M.T).max() <= 1e-12 * np.abs(M).max()
    np.linalg.cholesky((M + M.T) / 2)


def test_mg_vcycle_zero_off_fluid_and_linear(oracle_mod):
    O = oracle_mod
    n = (12, 10, 9)
    P = _params(O, n)
    t = S.random_mask(n, 0.6, 4).astype(np.uint8)
    rng = np.random.default_rng(4)
    r1, r2 = rng.normal(size=t.shape), rng.normal(size=t.shape)
    z1, z2 = O.mg_vcycle(P, t, r1), O.mg_vcycle(P, t, r2)
    z12 = O.mg_vcycle(P, t, 2.0 * r1 - 3.0 * r2)
    np.testing.assert_allclose(z12, 2.0 * z1 - 3.0 * z2, rtol=1e-11, atol=1e-12)
    assert np.all(z1[t == 0] == 0)


@pytest.mark.parametrize("n,seed", [((8, 8, 8), 7), ((13, 9, 11), 8)])
def test_pcg_mg_matches_dense_solve(oracle_mod, n, seed):
    O = oracle_mod
    P = _params(O, n, dt=1 / 240)
    t = S.random_mask(n, 0.7, seed).astype(np.uint8)
    rng = np.random.default_rng(seed)
    b = rng.normal(size=t.shape) * t
    x, it, rel = O.pcg_mg(P, t, b, tol=1e-13, max_iter=1000)
    assert it > 0 and rel <= 1e-13
    A, fl = _dense_A(O, P, t)
    xd = np.linalg.solve(A, b.ravel()[fl])
    assert np.linalg.norm(x.ravel()[fl] - xd) / np.linalg.norm(xd) <= 1e-10


@pytest.mark.parametrize("n,cap", [(32, 12), (64, 14)])
def test_pcg_mg_iterations_nearly_grid_independent(oracle_mod, n, cap):
    """The V-cycle makes the iteration count nearly independent of the grid (9 and 10
    at 32^3 and 64^3 to 1e-8, against 89 and 178 for Jacobi); a mis-scaled level or a
    lost correction shows up as many more iterations."""
    O = oracle_mod
    sc = S.dam_break(n)
    P = _params(O, n)
    r = O.step(P, *sc.arrays())
    _, it_j, _ = O.pcg(P, r.type, r.rhs, tol=1e-8, max_iter=5000)
    x, it_mg, rel = O.pcg_mg(P, r.type, r.rhs, tol=1e-8, max_iter=5000)
    assert 0 < it_mg <= cap and it_mg * 6 < it_j, (it_mg, it_j)
    xj, _, _ = O.pcg(P, r.type, r.rhs, tol=1e-13, max_iter=20000)
    assert np.linalg.norm(x - xj) <= 1e-6 * np.linalg.norm(xj)


# ------------------------------------------------------------ red-black Gauss-Seidel solver

@pytest.mark.parametrize("n,seed", [((6, 5, 4), 1), ((8, 8, 8), 2)])
def test_rbgs_matches_dense_solve(oracle_mod, n, seed):
    O = oracle_mod
    P = _params(O, n, dt=0.01, rho=2.0)
    t = S.random_mask(n, 0.6, seed).astype(np.uint8)
    A, fl = _dense_A(O, P, t)
    rng = np.random.default_rng(seed)
    b = np.zeros(t.shape)
    b.ravel()[fl] = rng.normal(size=fl.size)
    x, it, rel = O.rbgs(P, t, b, tol=1e-12, max_pairs=20000)
    assert it > 0 and it % 8 == 0 and rel <= 1e-12
    want = np.linalg.solve(A, b.ravel()[fl])
    assert np.abs(x.ravel()[fl] - want).max() <= 1e-9 * np.abs(want).max()


def test_rbgs_is_red_then_black_gauss_seidel(oracle_mod):
    """Eight sweep pairs equal the textbook Gauss-Seidel on the assembled matrix with
    the rows taken red (i+j+k even) first, then black."""
    O = oracle_mod
    n = (5, 4, 3)
    P = _params(O, n, dt=0.02, rho=1.0)
    t = S.random_mask(n, 0.7, 3).astype(np.uint8)
    A, fl = _dense_A(O, P, t)
    rng = np.random.default_rng(4)
    b = np.zeros(t.shape)
    b.ravel()[fl] = rng.normal(size=fl.size)
    x, it, _ = O.rbgs(P, t, b, tol=1e-300, max_pairs=8)
    assert it == -1
    k, j, i = np.unravel_index(fl, t.shape)
    red = ((i + j + k) % 2) == 0
    order = np.concatenate([np.flatnonzero(red), np.flatnonzero(~red)])
    y = np.zeros(fl.size)
    bb = b.ravel()[fl]
    for _ in range(8):
        for r in order:
            y[r] = (bb[r] - A[r] @ y + A[r, r] * y[r]) / A[r, r]
    assert np.abs(x.ravel()[fl] - y).max() <= 1e-12 * max(np.abs(y).max(), 1e-300)


def test_rbgs_cap_and_zero_rhs(oracle_mod):
    O = oracle_mod
    n = (6, 6, 6)
    P = _params(O, n)
    t = S.random_mask(n, 0.5, 7).astype(np.uint8)
    b = np.zeros(t.shape)
    x, it, rel = O.rbgs(P, t, b)
    assert it == 0 and not x.any()
    b.ravel()[np.flatnonzero(t.ravel())] = 1.0
    x, it, rel = O.rbgs(P, t, b, tol=1e-30, max_pairs=24)
    assert it == -1 and 0 < rel < 1


def test_oracle_thread_count_setter():
    """The single-thread timing of the bench's CPU baseline relies on the setter."""
    import oracle as O
    n0 = O.num_threads()
    try:
        O.set_num_threads(1)
        assert O.num_threads() == 1
    finally:
        O.set_num_threads(n0)
    assert O.num_threads() == n0
