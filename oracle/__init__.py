"""FP64 CPU oracle of the FLIP step (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  It wraps ``flip_oracle.c`` (compiled by
``oracle/build.py``) with numpy in/out; it shares nothing with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

_lib = None


class OracleParams(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("dx", C.c_double), ("dt", C.c_double),
                ("gravity", C.c_double * 3), ("rho", C.c_double), ("flip_ratio", C.c_double),
                ("skin", C.c_double), ("cg_tol", C.c_double), ("cg_max_iter", C.c_int32),
                ("advect_source", C.c_int32), ("preconditioner", C.c_int32), ("mg_nu", C.c_int32),
                ("mg_omega", C.c_double), ("cfl", C.c_double), ("ppc_min", C.c_int32),
                ("ppc_max", C.c_int32), ("reseed_seed", C.c_uint64), ("reseed_step", C.c_int64)]


class OracleStats(C.Structure):
    _fields_ = [("cg_iterations", C.c_int32), ("cg_rel_residual", C.c_double),
                ("rel_divergence", C.c_double), ("n_fluid", C.c_int64), ("dt", C.c_double),
                ("added", C.c_int64), ("removed", C.c_int64)]


class OracleFields(C.Structure):
    _fields_ = [("u_old", C.c_void_p * 3), ("u_star", C.c_void_p * 3), ("u_new", C.c_void_p * 3),
                ("pressure", C.c_void_p), ("rhs", C.c_void_p), ("type", C.c_void_p)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P = C.POINTER(OracleParams)
        vp = C.c_void_p
        L.oracle_n_cells.argtypes = [P]; L.oracle_n_cells.restype = C.c_int64
        L.oracle_n_faces.argtypes = [P, C.c_int]; L.oracle_n_faces.restype = C.c_int64
        L.oracle_hat.argtypes = [C.c_double]; L.oracle_hat.restype = C.c_double
        L.oracle_cell_of.argtypes = [P, C.c_double, C.c_double, C.c_double, vp]
        L.oracle_weight.argtypes = [P, C.c_int, C.c_int64, C.c_int64, C.c_int64,
                                    C.c_double, C.c_double, C.c_double]
        L.oracle_weight.restype = C.c_double
        L.oracle_bin.argtypes = [P, C.c_int64, vp, vp, vp, vp, vp]
        L.oracle_p2g.argtypes = [P, C.c_int, vp, vp, vp, vp, vp, vp, vp, vp]
        L.oracle_cell_types.argtypes = [P, vp, vp]
        L.oracle_forces_walls.argtypes = [P, C.c_int, vp, vp]
        L.oracle_divergence.argtypes = [P, vp, vp, vp]
        L.oracle_apply_A.argtypes = [P, vp, vp, vp]
        L.oracle_pcg.argtypes = [P, vp, vp, C.c_double, C.c_int, vp, vp]
        L.oracle_pcg.restype = C.c_int
        L.oracle_mg_levels.argtypes = [P, vp]
        L.oracle_mg_levels.restype = C.c_int
        L.oracle_mg_vcycle.argtypes = [P, vp, vp, vp, C.c_int, C.c_double]
        L.oracle_pcg_mg.argtypes = [P, vp, vp, C.c_double, C.c_int, C.c_int, C.c_double, vp, vp]
        L.oracle_pcg_mg.restype = C.c_int
        L.oracle_rbgs.argtypes = [P, vp, vp, C.c_double, C.c_int, vp, vp]
        L.oracle_rbgs.restype = C.c_int
        L.oracle_project.argtypes = [P, C.c_int, vp, vp, vp, vp]
        L.oracle_interp.argtypes = [P, C.c_int, vp, C.c_double, C.c_double, C.c_double]
        L.oracle_interp.restype = C.c_double
        L.oracle_g2p.argtypes = [P, C.c_int64, vp, vp, vp, vp, vp, vp, vp, vp]
        L.oracle_div_norm.argtypes = [P, vp, vp]; L.oracle_div_norm.restype = C.c_double
        L.oracle_step.argtypes = [P, C.c_int64, vp, vp, vp, vp, vp, vp,
                                  C.POINTER(OracleFields), C.POINTER(OracleStats)]
        L.oracle_step.restype = C.c_int
        L.oracle_step_ex.argtypes = [P, C.POINTER(C.c_int64), C.c_int64, vp, vp, vp, vp, vp, vp,
                                     C.POINTER(OracleFields), C.POINTER(OracleStats)]
        L.oracle_step_ex.restype = C.c_int
        L.oracle_num_threads.restype = C.c_int
        L.oracle_set_num_threads.argtypes = [C.c_int]
        L.oracle_set_num_threads.restype = None
        L.oracle_energy.argtypes = [C.c_int64, vp, vp, vp, vp, vp, vp, vp, C.c_double, vp]
        L.oracle_energy.restype = None
        L.oracle_blobby_kernel.argtypes = [C.c_double]
        L.oracle_blobby_kernel.restype = C.c_double
        L.oracle_sdf.argtypes = [C.c_int64, vp, vp, vp, vp, vp, C.c_double, C.c_double,
                                 C.c_double, vp]
        L.oracle_sdf.restype = None
        L.oracle_mc_count.argtypes = [vp, vp, C.c_double, vp]
        L.oracle_mc_count.restype = C.c_int64
        L.oracle_mc.argtypes = [vp, vp, C.c_double, vp, C.c_double, vp, vp, vp, vp]
        L.oracle_mc.restype = None
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


@dataclass
class Params:
    """Physical and solver parameters of one scene (plain values)."""

    n: tuple = (32, 32, 32)
    dx: float = 1.0 / 32
    dt: float = 1.0 / 240
    gravity: tuple = (0.0, -9.81, 0.0)
    rho: float = 1.0
    flip_ratio: float = 0.95
    skin: float | None = None  # default 1e-3 * dx
    cg_tol: float = 1e-6
    cg_max_iter: int = 0       # default 20 * max(n)
    advect_source: int = 0
    preconditioner: int = 1    # 0 Jacobi, 1 multigrid V-cycle
    mg_nu: int = 2
    mg_omega: float = 2.0
    cfl: float = 0.0           # Sec. 3.1.4 CFL number; 0: fixed dt
    ppc_min: int = 0           # Sec. 3.1.2 reseeding bounds (0: off)
    ppc_max: int = 0
    reseed_seed: int = 0

    def c(self) -> OracleParams:
        p = OracleParams()
        for a in range(3):
            p.n[a] = int(self.n[a])
            p.gravity[a] = float(self.gravity[a])
        p.dx, p.dt, p.rho = float(self.dx), float(self.dt), float(self.rho)
        p.flip_ratio = float(self.flip_ratio)
        p.skin = float(1e-3 * self.dx if self.skin is None else self.skin)
        p.cg_tol = float(self.cg_tol)
        p.cg_max_iter = int(self.cg_max_iter or 20 * max(self.n))
        p.advect_source = int(self.advect_source)
        p.preconditioner = int(self.preconditioner)
        p.mg_nu = int(self.mg_nu)
        p.mg_omega = float(self.mg_omega)
        p.cfl = float(self.cfl)
        p.ppc_min = int(self.ppc_min)
        p.ppc_max = int(self.ppc_max)
        p.reseed_seed = int(self.reseed_seed)
        return p


def face_shape(n, comp):
    """(nz', ny', nx') shape of a component's face array (one extra node on its own axis)."""
    nx, ny, nz = n
    return (nz + (comp == 2), ny + (comp == 1), nx + (comp == 0))


def cell_shape(n):
    return (n[2], n[1], n[0])


@dataclass
class StepResult:
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    u: np.ndarray
    v: np.ndarray
    w: np.ndarray
    u_old: list = field(default_factory=list)
    u_star: list = field(default_factory=list)
    u_new: list = field(default_factory=list)
    pressure: np.ndarray | None = None
    rhs: np.ndarray | None = None
    type: np.ndarray | None = None
    status: int = 0
    cg_iterations: int = 0
    cg_rel_residual: float = 0.0
    rel_divergence: float = 0.0
    n_fluid: int = 0
    dt: float = 0.0
    added: int = 0
    removed: int = 0


def step(params: Params, x, y, z, u, v, w, fields: bool = True, step_index: int = 0,
         capacity: int | None = None) -> StepResult:
    """One oracle step; particle arrays are copied to float64 and returned in the same
    order (with reseeding: the survivors in order, then the new particles)."""
    L = lib()
    P = params.c()
    P.reseed_step = int(step_index)
    reseed = params.ppc_min > 0 or params.ppc_max > 0
    np_ = int(np.asarray(x).shape[0])
    cap = np_ if not reseed else (capacity or np_ + params.ppc_min * int(np.prod(params.n)))
    arrs = []
    for a in (x, y, z, u, v, w):
        buf = np.zeros(cap, dtype=np.float64)
        buf[:np_] = a
        arrs.append(buf)
    res = StepResult(*arrs)
    F = OracleFields()
    if fields:
        res.u_old = [np.zeros(face_shape(params.n, d)) for d in range(3)]
        res.u_star = [np.zeros(face_shape(params.n, d)) for d in range(3)]
        res.u_new = [np.zeros(face_shape(params.n, d)) for d in range(3)]
        res.pressure = np.zeros(cell_shape(params.n))
        res.rhs = np.zeros(cell_shape(params.n))
        res.type = np.zeros(cell_shape(params.n), np.uint8)
        for d in range(3):
            F.u_old[d] = res.u_old[d].ctypes.data
            F.u_star[d] = res.u_star[d].ctypes.data
            F.u_new[d] = res.u_new[d].ctypes.data
        F.pressure = res.pressure.ctypes.data
        F.rhs = res.rhs.ctypes.data
        F.type = res.type.ctypes.data
    S = OracleStats()
    if reseed:
        n_io = C.c_int64(np_)
        res.status = L.oracle_step_ex(C.byref(P), C.byref(n_io), cap, *[_p(a) for a in arrs],
                                      C.byref(F) if fields else None, C.byref(S))
        for name, a in zip(("x", "y", "z", "u", "v", "w"), arrs):
            setattr(res, name, a[:n_io.value].copy())
    else:
        res.status = L.oracle_step(C.byref(P), np_, *[_p(a) for a in arrs],
                                   C.byref(F) if fields else None, C.byref(S))
    res.cg_iterations = S.cg_iterations
    res.cg_rel_residual = S.cg_rel_residual
    res.rel_divergence = S.rel_divergence
    res.n_fluid = S.n_fluid
    res.dt = S.dt
    res.added = S.added
    res.removed = S.removed
    return res


def bin_particles(params: Params, x, y, z):
    L = lib()
    P = params.c()
    x, y, z = (np.ascontiguousarray(a, np.float64) for a in (x, y, z))
    nc = int(np.prod(params.n))
    start = np.zeros(nc + 1, np.int64)
    order = np.zeros(max(x.shape[0], 1), np.int64)
    L.oracle_bin(C.byref(P), x.shape[0], _p(x), _p(y), _p(z), _p(start), _p(order))
    return start, order[:x.shape[0]]


def p2g(params: Params, comp, x, y, z, vel):
    """Gather-form P2G of one component; returns (grid, weight_sum) on the face array."""
    L = lib()
    P = params.c()
    x, y, z, vel = (np.ascontiguousarray(a, np.float64) for a in (x, y, z, vel))
    start, order = bin_particles(params, x, y, z)
    grid = np.zeros(face_shape(params.n, comp))
    ws = np.zeros(face_shape(params.n, comp))
    L.oracle_p2g(C.byref(P), comp, _p(x), _p(y), _p(z), _p(vel), _p(start), _p(order),
                 _p(grid), _p(ws))
    return grid, ws


def cell_types(params: Params, x, y, z):
    start, _ = bin_particles(params, x, y, z)
    t = np.zeros(cell_shape(params.n), np.uint8)
    lib().oracle_cell_types(C.byref(params.c()), _p(start), _p(t))
    return t


def forces_walls(params: Params, comp, u_old):
    u_old = np.ascontiguousarray(u_old, np.float64)
    out = np.zeros_like(u_old)
    lib().oracle_forces_walls(C.byref(params.c()), comp, _p(u_old), _p(out))
    return out


def divergence(params: Params, u3, type_):
    u3 = [np.ascontiguousarray(a, np.float64) for a in u3]
    type_ = np.ascontiguousarray(type_, np.uint8)
    arr = (C.c_void_p * 3)(*[a.ctypes.data for a in u3])
    b = np.zeros(cell_shape(params.n))
    lib().oracle_divergence(C.byref(params.c()), arr, _p(type_), _p(b))
    return b


def apply_A(params: Params, type_, p):
    type_ = np.ascontiguousarray(type_, np.uint8)
    p = np.ascontiguousarray(p, np.float64)
    out = np.zeros_like(p)
    lib().oracle_apply_A(C.byref(params.c()), _p(type_), _p(p), _p(out))
    return out


def pcg(params: Params, type_, b, tol=None, max_iter=None):
    type_ = np.ascontiguousarray(type_, np.uint8)
    b = np.ascontiguousarray(b, np.float64)
    x = np.zeros_like(b)
    rel = C.c_double(0.0)
    P = params.c()
    it = lib().oracle_pcg(C.byref(P), _p(type_), _p(b), P.cg_tol if tol is None else tol,
                          P.cg_max_iter if max_iter is None else max_iter, _p(x), C.byref(rel))
    return x, it, rel.value


def mg_levels(params: Params):
    dims = np.zeros((12, 3), np.int32)
    L = lib().oracle_mg_levels(C.byref(params.c()), _p(dims))
    return [tuple(int(v) for v in dims[l]) for l in range(L)]


MG_NU = 2        # red-black sweep pairs before and after the coarse correction
MG_OMEGA = 2.0   # over-correction of the coarse correction


def mg_vcycle(params: Params, type_, r, nu=MG_NU, omega=MG_OMEGA):
    type_ = np.ascontiguousarray(type_, np.uint8)
    r = np.ascontiguousarray(r, np.float64)
    z = np.zeros_like(r)
    lib().oracle_mg_vcycle(C.byref(params.c()), _p(type_), _p(r), _p(z), int(nu), float(omega))
    return z


def pcg_mg(params: Params, type_, b, tol=None, max_iter=None, nu=MG_NU, omega=MG_OMEGA):
    type_ = np.ascontiguousarray(type_, np.uint8)
    b = np.ascontiguousarray(b, np.float64)
    x = np.zeros_like(b)
    rel = C.c_double(0.0)
    P = params.c()
    it = lib().oracle_pcg_mg(C.byref(P), _p(type_), _p(b), P.cg_tol if tol is None else tol,
                             P.cg_max_iter if max_iter is None else max_iter, int(nu),
                             float(omega), _p(x), C.byref(rel))
    return x, it, rel.value


def rbgs(params: Params, type_, b, tol=None, max_pairs=None):
    """Red-black Gauss-Seidel as the solver (Sec. 3.2.3): (x, pairs or -1, rel)."""
    L = lib()
    P = params.c()
    t = np.ascontiguousarray(type_, np.uint8)
    bb = np.ascontiguousarray(b, np.float64)
    x = np.zeros_like(bb)
    rel = C.c_double(0.0)
    it = L.oracle_rbgs(C.byref(P), _p(t), _p(bb), float(params.cg_tol if tol is None else tol),
                       int(P.cg_max_iter if max_pairs is None else max_pairs), _p(x), C.byref(rel))
    return x, it, rel.value


def project(params: Params, comp, u_star, p, type_):
    u_star = np.ascontiguousarray(u_star, np.float64)
    p = np.ascontiguousarray(p, np.float64)
    type_ = np.ascontiguousarray(type_, np.uint8)
    out = np.zeros_like(u_star)
    lib().oracle_project(C.byref(params.c()), comp, _p(u_star), _p(p), _p(type_), _p(out))
    return out


def interp(params: Params, comp, fieldarr, x, y, z):
    fieldarr = np.ascontiguousarray(fieldarr, np.float64)
    L = lib()
    P = params.c()
    return np.array([L.oracle_interp(C.byref(P), comp, _p(fieldarr), float(a), float(b), float(c))
                     for a, b, c in zip(np.atleast_1d(x), np.atleast_1d(y), np.atleast_1d(z))])


def g2p(params: Params, x, y, z, u, v, w, u_old3, u_new3):
    arrs = [np.array(a, dtype=np.float64, copy=True) for a in (x, y, z, u, v, w)]
    uo = [np.ascontiguousarray(a, np.float64) for a in u_old3]
    un = [np.ascontiguousarray(a, np.float64) for a in u_new3]
    A = (C.c_void_p * 3)(*[a.ctypes.data for a in uo])
    B = (C.c_void_p * 3)(*[a.ctypes.data for a in un])
    lib().oracle_g2p(C.byref(params.c()), arrs[0].shape[0], *[_p(a) for a in arrs], A, B)
    return arrs


def div_norm(params: Params, u3, type_):
    u3 = [np.ascontiguousarray(a, np.float64) for a in u3]
    type_ = np.ascontiguousarray(type_, np.uint8)
    arr = (C.c_void_p * 3)(*[a.ctypes.data for a in u3])
    return lib().oracle_div_norm(C.byref(params.c()), arr, _p(type_))


def weight(params: Params, comp, node, x, y, z):
    return lib().oracle_weight(C.byref(params.c()), comp, int(node[0]), int(node[1]),
                               int(node[2]), float(x), float(y), float(z))


def hat(r):
    return lib().oracle_hat(float(r))


def cell_of(params: Params, x, y, z):
    out = np.zeros(3, np.int64)
    lib().oracle_cell_of(C.byref(params.c()), float(x), float(y), float(z), _p(out))
    return out


def energy(gravity, mass, x, y, z, u, v, w):
    """(kinetic, potential, total) of a particle set of equal masses (Sec. 4, Fig. 10)."""
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (x, y, z, u, v, w)]
    g = np.asarray(gravity, dtype=np.float64)
    out = np.zeros(3)
    lib().oracle_energy(arrs[0].shape[0], *[_p(a) for a in arrs], _p(g), float(mass), _p(out))
    return tuple(float(t) for t in out)


def blobby_kernel(s: float) -> float:
    """k(s) = max(0, (1 - s^2)^3) of Sec. 3.3.1."""
    return float(lib().oracle_blobby_kernel(float(s)))


def sdf(x, y, z, n, origin, h, radius, search_radius):
    """Sec. 3.3.1 scalar field at the (n+1)^3 sampling corners; shape (nz+1, ny+1, nx+1)."""
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (x, y, z)]
    n3 = np.asarray(n, dtype=np.int32)
    o = np.asarray(origin, dtype=np.float64)
    phi = np.zeros((n3[2] + 1, n3[1] + 1, n3[0] + 1))
    lib().oracle_sdf(arrs[0].shape[0], *[_p(a) for a in arrs], _p(n3), _p(o), float(h),
                     float(radius), float(search_radius), _p(phi))
    return phi


@dataclass
class Mesh:
    vertices: np.ndarray   # (nv, 3) float64
    normals: np.ndarray    # (nv, 3)
    triangles: np.ndarray  # (nt, 3) int32
    vertex_edge: np.ndarray  # (nv,) int64


def marching_cubes(phi, origin, h, iso=0.0) -> Mesh:
    """Sec. 3.3.2 on a corner field of shape (nz+1, ny+1, nx+1)."""
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    n3 = np.array([phi.shape[2] - 1, phi.shape[1] - 1, phi.shape[0] - 1], dtype=np.int32)
    o = np.asarray(origin, dtype=np.float64)
    nt = C.c_int64(0)
    L = lib()
    nv = L.oracle_mc_count(_p(n3), _p(phi), float(iso), C.byref(nt))
    m = Mesh(np.zeros((nv, 3)), np.zeros((nv, 3)), np.zeros((nt.value, 3), np.int32),
             np.zeros(nv, np.int64))
    L.oracle_mc(_p(n3), _p(o), float(h), _p(phi), float(iso), _p(m.vertices), _p(m.vertex_edge),
                _p(m.triangles), _p(m.normals))
    return m


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def set_num_threads(n: int) -> None:
    """Threads for the oracle's later OpenMP regions (for single-thread timings)."""
    lib().oracle_set_num_threads(int(n))
