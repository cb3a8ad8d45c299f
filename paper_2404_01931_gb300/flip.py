"""Thin ctypes binding of the C ABI in include/flip.h (libflip_gb300.so).

The functions keep the C names (flip_create, flip_step, flip_read, ...) and only
marshal arguments: numpy arrays are host buffers, torch tensors on a CUDA
device are device buffers.  Every step of the FLIP pipeline runs in the
library's CUDA kernels; there is no Python or CPU fallback.  If the shared
library has not been built, importing works but the first call raises.

PyTorch supplies device memory (its caching allocator, through the library's
allocator hook) and streams.
"""
from __future__ import annotations

import ctypes as C
import os
import warnings

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libflip_gb300.so")

FLIP_OK = 0
FLIP_E_ARG = 1
FLIP_E_OOM = 2
FLIP_E_CUDA = 3
FLIP_E_NOT_CONVERGED = 4
FLIP_E_TIMEOUT = 5
FLIP_E_SIZE = 6
FLIP_E_NOGPU = 7
FLIP_E_CAPACITY = 8

FLIP_PREC_FP32 = 0
FLIP_PREC_MIXED_IR = 1
FLIP_ADVECT_PARTICLE = 0
FLIP_ADVECT_GRID = 1
FLIP_PRECOND_JACOBI = 0
FLIP_PRECOND_MG = 1
FLIP_PRECOND_RBGS = 2

(PX, PY, PZ, PU, PV, PW, PID, U_OLD, V_OLD, W_OLD, U_NEW, V_NEW, W_NEW, PRESSURE,
 PRESSURE_F64, RHS, CELL_TYPE) = range(17)
FIELD_DTYPE = {PX: np.float32, PY: np.float32, PZ: np.float32, PU: np.float32, PV: np.float32,
               PW: np.float32, PID: np.int32, U_OLD: np.float32, V_OLD: np.float32,
               W_OLD: np.float32, U_NEW: np.float32, V_NEW: np.float32, W_NEW: np.float32,
               PRESSURE: np.float32, PRESSURE_F64: np.float64, RHS: np.float32,
               CELL_TYPE: np.uint8}


class FlipError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"[{code}] {message}")
        self.code = code


class FlipParams(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("dx", C.c_double), ("dt", C.c_double),
                ("gravity", C.c_double * 3), ("rho", C.c_double), ("flip_ratio", C.c_double),
                ("skin", C.c_double), ("cg_tol", C.c_double), ("ir_tol", C.c_double),
                ("cg_max_iter", C.c_int32), ("ir_max_iter", C.c_int32),
                ("precision", C.c_int32), ("advect_source", C.c_int32),
                ("preconditioner", C.c_int32), ("mg_smooth", C.c_int32),
                ("warm_start", C.c_int32), ("cfl", C.c_double), ("ppc_min", C.c_int32),
                ("ppc_max", C.c_int32), ("max_particles", C.c_int64),
                ("reseed_seed", C.c_uint64)]


class FlipStats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("n_particles", C.c_int64), ("n_fluid_cells", C.c_int64),
                ("n_active_bricks", C.c_int64), ("cg_iterations", C.c_int64),
                ("ir_iterations", C.c_int32), ("kernel_launches", C.c_int32),
                ("cg_rel_residual", C.c_double), ("rel_divergence", C.c_double),
                ("max_speed", C.c_double), ("ms_bin", C.c_double), ("ms_p2g", C.c_double),
                ("ms_divergence", C.c_double), ("ms_pcg", C.c_double), ("ms_g2p", C.c_double),
                ("ms_total", C.c_double), ("dt_last", C.c_double),
                ("particles_added", C.c_int64), ("particles_removed", C.c_int64)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class RequestInfo(C.Structure):
    _fields_ = [("scene", C.c_int32), ("status", C.c_int32), ("t_arrival", C.c_double),
                ("t_start", C.c_double), ("t_done", C.c_double), ("batch_size", C.c_int32),
                ("reserved", C.c_int32)]


_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)


class FlipSurfaceParams(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("origin", C.c_double * 3), ("h", C.c_double),
                ("radius", C.c_double), ("search_radius", C.c_double), ("iso", C.c_double)]


SURF_FIELD, SURF_VERTICES, SURF_NORMALS, SURF_TRIANGLES, SURF_VERTEX_EDGE = range(5)
SURF_MAX_TRI = 12


class FlipAlloc(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("alloc", _ALLOC_FN), ("free", _FREE_FN)]


_lib = None


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libflip_gb300.so is not built ({LIB_PATH}); run "
                               "__graft_entry__.build() or paper_2404_01931_gb300/build_lib.py")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t
        PP = C.POINTER(FlipParams)
        L.flip_abi_version.restype = C.c_int
        L.flip_default_params.argtypes = [PP, i32, i32, i32]
        L.flip_default_params.restype = None
        L.flip_create.argtypes = [PP, vp, vp, vp, vp, vp, vp, i64, i32, C.POINTER(FlipAlloc), vp,
                                  C.POINTER(vp)]
        L.flip_step.argtypes = [vp, i32, C.POINTER(FlipStats)]
        L.flip_sync.argtypes = [vp]
        L.flip_read.argtypes = [vp, C.c_int, vp, sz, i32]
        L.flip_write.argtypes = [vp, C.c_int, vp, sz, i32]
        L.flip_read_particles.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, i32]
        L.flip_write_particles.argtypes = [vp, vp, vp, vp, vp, vp, vp, i32]
        L.flip_field_bytes.argtypes = [vp, C.c_int]
        L.flip_field_bytes.restype = sz
        L.flip_destroy.argtypes = [vp]
        L.flip_destroy.restype = None
        L.flip_strerror.argtypes = [C.c_int]
        L.flip_strerror.restype = C.c_char_p
        L.flip_last_error.restype = C.c_char_p
        L.flip_solve_pressure.argtypes = [PP, vp, vp, vp, vp, C.POINTER(i32),
                                          C.POINTER(C.c_double)]
        L.flip_batch_create.argtypes = [i32, vp, C.POINTER(vp)]
        L.flip_batch_step.argtypes = [vp, C.POINTER(vp), i32, i32, C.POINTER(FlipStats)]
        L.flip_batch_destroy.argtypes = [vp]
        L.flip_batch_destroy.restype = None
        L.flip_footprint_bytes.argtypes = [PP, i64]
        L.flip_footprint_bytes.restype = sz
        L.flip_server_create.argtypes = [sz, i32, C.POINTER(vp)]
        L.flip_server_add_scene.argtypes = [vp, PP, vp, vp, vp, vp, vp, vp, i64, C.POINTER(i32)]
        L.flip_server_submit.argtypes = [vp, i32, C.c_double, C.POINTER(i64)]
        L.flip_server_wait.argtypes = [vp, i64, C.POINTER(RequestInfo)]
        L.flip_server_drain.argtypes = [vp]
        L.flip_server_now.argtypes = [vp]
        L.flip_server_now.restype = C.c_double
        L.flip_server_usage.argtypes = [vp, C.POINTER(i32), C.POINTER(sz)]
        L.flip_server_scene_handle.argtypes = [vp, i32, C.POINTER(vp)]
        L.flip_server_remove_scene.argtypes = [vp, i32]
        L.flip_server_destroy.argtypes = [vp]
        L.flip_server_destroy.restype = None
        L.flip_solve_pressure_noalloc.argtypes = [PP, vp, vp, vp, vp, C.POINTER(i32),
                                                  C.POINTER(C.c_double)]
        L.flip_energy.argtypes = [vp, C.c_double, C.POINTER(C.c_double)]
        L.flip_set_solver_blocks.argtypes = [vp, i32]
        L.flip_autotune_solver.argtypes = [vp, i32, C.POINTER(i32)]
        L.flip_set_transfer_ctas.argtypes = [vp, i32, i32]
        L.flip_get_transfer_ctas.argtypes = [vp, C.POINTER(i32), C.POINTER(i32)]
        L.flip_autotune_transfers.argtypes = [vp, i32, C.POINTER(i32), C.POINTER(i32)]
        L.flip_batch_set_team_exponent.argtypes = [vp, C.c_double]
        L.flip_batch_graph_active.argtypes = [vp]
        L.flip_batch_set_graphs.argtypes = [vp, i32]
        L.flip_batch_autotune.argtypes = [vp, C.POINTER(vp), i32, i32, C.POINTER(C.c_double)]
        SP = C.POINTER(FlipSurfaceParams)
        L.flip_surface_default_params.argtypes = [PP, SP]
        L.flip_surface_default_params.restype = None
        L.flip_surface_create.argtypes = [SP, vp, C.POINTER(vp)]
        L.flip_surface_sdf.argtypes = [vp, vp]
        L.flip_surface_set_field.argtypes = [vp, vp, i32]
        L.flip_surface_mesh.argtypes = [vp, C.POINTER(i64), C.POINTER(i64)]
        L.flip_surface_bytes.argtypes = [vp, C.c_int]
        L.flip_surface_bytes.restype = sz
        L.flip_surface_read.argtypes = [vp, C.c_int, vp, sz, i32]
        L.flip_surface_destroy.argtypes = [vp]
        L.flip_surface_destroy.restype = None
        L.flip_surface_case_table.argtypes = [vp, vp]
        L.flip_server_set_overlap.argtypes = [vp, i32]
        L.flip_server_set_fused.argtypes = [vp, i32]
        L.flip_batch_set_fused.argtypes = [vp, i32]
        L.flip_batch_get_form.argtypes = [vp, C.POINTER(i32), C.POINTER(i32)]
        L.flip_step_times.argtypes = [vp, vp, i32]
        L.flip_step_times.restype = i32
        L.flip_set_wait_timeout.argtypes = [vp, C.c_uint64]
        L.flip_dot_f32.argtypes = [vp, vp, i64, C.POINTER(C.c_double), vp]
        L.flip_residual_pairs.argtypes = [PP, vp, vp, vp, vp, vp, vp, vp, vp]
        if L.flip_abi_version() != 5:
            raise RuntimeError("libflip_gb300 ABI version mismatch")
        _lib = L
    return _lib


def last_error() -> str:
    return lib().flip_last_error().decode()


def _check(rc: int, allow=(FLIP_OK,)) -> int:
    if rc in allow:
        return rc
    if rc in (FLIP_E_NOT_CONVERGED, FLIP_E_CAPACITY):
        warnings.warn(f"flip: {last_error()}", RuntimeWarning, stacklevel=3)
        return rc
    raise FlipError(rc, f"{lib().flip_strerror(rc).decode()}: {last_error()}")


def _buf(a, dtype):
    """(pointer, nbytes, is_device, keepalive) of a numpy array or torch tensor."""
    if isinstance(a, np.ndarray):
        if a.dtype != dtype or not a.flags.c_contiguous:
            raise TypeError(f"expected a C-contiguous {np.dtype(dtype).name} array")
        return a.ctypes.data, a.nbytes, 0, a
    import torch
    if isinstance(a, torch.Tensor):
        want = {np.float32: torch.float32, np.float64: torch.float64, np.int32: torch.int32,
                np.uint8: torch.uint8}[np.dtype(dtype).type]
        if a.dtype != want or not a.is_contiguous():
            raise TypeError(f"expected a contiguous {want} tensor")
        return a.data_ptr(), a.numel() * a.element_size(), int(a.is_cuda), a
    raise TypeError(f"unsupported buffer type {type(a)}")


def default_params(nx: int, ny: int | None = None, nz: int | None = None, **overrides) -> FlipParams:
    p = FlipParams()
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    lib().flip_default_params(C.byref(p), nx, ny, nz)
    for k, v in overrides.items():
        if k in ("n", "gravity"):
            for i in range(3):
                getattr(p, k)[i] = v[i]
        else:
            setattr(p, k, v)
    return p


class _TorchAllocator:
    """Allocator hook backed by PyTorch's CUDA caching allocator."""

    def __init__(self, device: int):
        import torch
        self.device = device
        self._torch = torch

        def _alloc(ctx, nbytes, stream):
            try:
                return self._torch.cuda.caching_allocator_alloc(int(nbytes), self.device,
                                                                int(stream or 0))
            except Exception:  # out of memory: the library reports FLIP_E_OOM
                return None

        def _free(ctx, ptr, nbytes, stream):
            try:
                self._torch.cuda.caching_allocator_delete(int(ptr))
            except Exception:
                pass

        self._fa = _ALLOC_FN(_alloc)
        self._ff = _FREE_FN(_free)
        self.struct = FlipAlloc(None, self._fa, self._ff)


def flip_create(params: FlipParams, x, y, z, u, v, w, stream=None, allocator="torch"):
    """Returns (handle, keepalive) for a new scene; see flip_create in include/flip.h."""
    bufs = [_buf(a, np.float32) for a in (x, y, z, u, v, w)]
    np_ = bufs[0][1] // 4
    if any(b[1] != bufs[0][1] for b in bufs) or len({b[2] for b in bufs}) != 1:
        raise ValueError("particle arrays must have one length and live on one side")
    keep = [b[3] for b in bufs]
    alloc_ptr = None
    if allocator == "torch":
        import torch
        if torch.cuda.is_available():
            ta = _TorchAllocator(torch.cuda.current_device())
            keep.append(ta)
            alloc_ptr = C.byref(ta.struct)
    elif allocator is not None:
        # any object holding a FlipAlloc in .struct (callbacks kept alive by it)
        if not isinstance(getattr(allocator, "struct", None), FlipAlloc):
            raise ValueError("allocator must be 'torch', None or an object with a FlipAlloc "
                             ".struct")
        keep.append(allocator)
        alloc_ptr = C.byref(allocator.struct)
    h = C.c_void_p()
    rc = lib().flip_create(C.byref(params), *[C.c_void_p(b[0]) for b in bufs], np_, bufs[0][2],
                           alloc_ptr, C.c_void_p(stream or 0), C.byref(h))
    _check(rc)
    return h, keep


def flip_step(h, nsteps: int = 1, stats: bool = False):
    """Advances nsteps; returns (status, FlipStats or None)."""
    st = FlipStats() if stats else None
    rc = lib().flip_step(h, int(nsteps), C.byref(st) if stats else None)
    return _check(rc), st


def flip_sync(h) -> int:
    return _check(lib().flip_sync(h))


def flip_field_bytes(h, field: int) -> int:
    return int(lib().flip_field_bytes(h, field))


def flip_read(h, field: int, out=None):
    """Reads a field into out (numpy or torch); allocates a numpy array if out is None."""
    dtype = FIELD_DTYPE[field]
    if out is None:
        out = np.empty(flip_field_bytes(h, field) // np.dtype(dtype).itemsize, dtype)
    ptr, nbytes, dev, _ = _buf(out, dtype)
    _check(lib().flip_read(h, field, C.c_void_p(ptr), nbytes, dev))
    return out


def flip_write(h, field: int, src):
    ptr, nbytes, dev, _ = _buf(src, FIELD_DTYPE[field])
    _check(lib().flip_write(h, field, C.c_void_p(ptr), nbytes, dev))


def flip_read_particles(h, x, y, z, u, v, w, ids=None):
    """Reads the six particle arrays (and ids) into caller buffers (numpy or torch)."""
    bufs = [_buf(a, np.float32) for a in (x, y, z, u, v, w)]
    idb = _buf(ids, np.int32) if ids is not None else None
    _check_particle_sizes(h, bufs + ([idb] if idb else []))
    dev = bufs[0][2]
    _check(lib().flip_read_particles(h, *[C.c_void_p(b[0]) for b in bufs],
                                     C.c_void_p(idb[0]) if idb else None, dev))


def _check_particle_sizes(h, bufs):
    """Every buffer must hold the current particle count (it varies with reseeding)."""
    need = lib().flip_field_bytes(h, PX)
    for b in bufs:
        if b[1] != need:
            raise ValueError(f"particle buffer of {b[1]} bytes; the handle holds {need // 4} "
                             "particles")


def flip_write_particles(h, x, y, z, u, v, w):
    bufs = [_buf(a, np.float32) for a in (x, y, z, u, v, w)]
    _check_particle_sizes(h, bufs)
    _check(lib().flip_write_particles(h, *[C.c_void_p(b[0]) for b in bufs], bufs[0][2]))


def flip_energy(h, particle_mass: float):
    """(kinetic, potential, total) energy of the handle's particles (Sec. 4, Fig. 10)."""
    out = (C.c_double * 3)()
    _check(lib().flip_energy(h, float(particle_mass), out))
    return float(out[0]), float(out[1]), float(out[2])


def flip_destroy(h):
    if h:
        lib().flip_destroy(h)


def _grid_cells(params: FlipParams) -> int:
    return int(params.n[0]) * int(params.n[1]) * int(params.n[2])


def _solve_buffers(params: FlipParams, type_, b, p, name: str):
    """Device pointers of the solve's arrays, each checked to hold one entry per
    cell of params.n (the library reads and writes that many)."""
    tp, tn, tdev, _ = _buf(type_, np.uint8)
    bp, bn, bdev, _ = _buf(b, np.float32)
    pp, pn, pdev, _ = _buf(p, np.float32)
    nc = _grid_cells(params)
    if tn != nc or bn != 4 * nc or pn != 4 * nc:
        raise FlipError(FLIP_E_SIZE, f"{name}: type, b and p must hold {nc} cells each "
                                     f"(got {tn}, {bn // 4}, {pn // 4})")
    if not (tdev and bdev and pdev):
        raise ValueError(f"{name} takes device buffers")
    return tp, bp, pp


def flip_solve_pressure(params: FlipParams, type_, b, p, stream=None):
    """A p = b on device tensors (uint8 types, float32 b and p); returns (status, iters, rel)."""
    tp, bp, pp = _solve_buffers(params, type_, b, p, "flip_solve_pressure")
    it = C.c_int32(0)
    rel = C.c_double(0.0)
    rc = lib().flip_solve_pressure(C.byref(params), C.c_void_p(tp), C.c_void_p(bp),
                                   C.c_void_p(pp), C.c_void_p(stream or 0), C.byref(it),
                                   C.byref(rel))
    return _check(rc), it.value, rel.value


def flip_solve_pressure_noalloc(params: FlipParams, type_, b, p, stream=None):
    """As flip_solve_pressure, with no device allocation: for callers that cannot
    allocate while they run (memory owned by a host application's allocator, or
    loops where cudaMalloc/cudaFree may not synchronise the device).  Grids up to
    FLIP_NOALLOC_MAX_CELLS cells.  Returns (status, iterations, rel_residual)."""
    tp, bp, pp = _solve_buffers(params, type_, b, p, "flip_solve_pressure_noalloc")
    it = C.c_int32(0)
    rel = C.c_double(0.0)
    rc = lib().flip_solve_pressure_noalloc(C.byref(params), C.c_void_p(tp), C.c_void_p(bp),
                                           C.c_void_p(pp), C.c_void_p(stream or 0),
                                           C.byref(it), C.byref(rel))
    return _check(rc), it.value, rel.value


FLIP_NOALLOC_MAX_CELLS = 262144


def flip_dot_f32(a, b, stream=None) -> float:
    """sum a[i] b[i] of two float32 device tensors by the CG's reduction (float
    pairs per thread, warp and CTA; FP64 at the end)."""
    ap, an, adev, _ = _buf(a, np.float32)
    bp, bn, bdev, _ = _buf(b, np.float32)
    if an != bn:
        raise FlipError(FLIP_E_SIZE, "a and b must have one length")
    if an and not (adev and bdev):
        raise ValueError("flip_dot_f32 takes device buffers")
    out = C.c_double(0.0)
    _check(lib().flip_dot_f32(C.c_void_p(ap), C.c_void_p(bp), an // 4, C.byref(out),
                              C.c_void_p(stream or 0)))
    return float(out.value)


def flip_residual_pairs(params: FlipParams, type_, x_hi, x_lo, b_hi, b_lo, r_hi, r_lo,
                        stream=None):
    """r = b - A x in float pairs on the grid of params (the mixed-mode refinement's
    residual); every array is a device tensor with one entry per cell."""
    nc = _grid_cells(params)
    tp, tn, tdev, _ = _buf(type_, np.uint8)
    fl = [_buf(a, np.float32) for a in (x_hi, x_lo, b_hi, b_lo, r_hi, r_lo)]
    if tn != nc or any(f[1] != 4 * nc for f in fl):
        raise FlipError(FLIP_E_SIZE, f"flip_residual_pairs: every array must hold {nc} cells")
    if not (tdev and all(f[2] for f in fl)):
        raise ValueError("flip_residual_pairs takes device buffers")
    _check(lib().flip_residual_pairs(C.byref(params), C.c_void_p(tp),
                                     *[C.c_void_p(f[0]) for f in fl], C.c_void_p(stream or 0)))


def flip_batch_create(capacity: int, stream=None):
    b = C.c_void_p()
    _check(lib().flip_batch_create(int(capacity), C.c_void_p(stream or 0), C.byref(b)))
    return b


def flip_batch_step(b, handles, nsteps: int = 1, stats: bool = False):
    """Advances the scenes (handles) together; returns (status, [FlipStats] or None)."""
    n = len(handles)
    arr = (C.c_void_p * max(n, 1))(*[h.value if isinstance(h, C.c_void_p) else h for h in handles])
    st = (FlipStats * max(n, 1))() if stats else None
    rc = lib().flip_batch_step(b, arr, n, int(nsteps), st)
    return _check(rc), (list(st)[:n] if stats else None)


def flip_batch_destroy(b):
    if b:
        lib().flip_batch_destroy(b)


class Batch:
    """Batch runner: advances several Simulations together (see flip_batch_step)."""

    def __init__(self, capacity: int, stream=None):
        self.b = flip_batch_create(capacity, stream)

    def step(self, sims, nsteps: int = 1, stats: bool = False):
        return flip_batch_step(self.b, [s.h for s in sims], nsteps, stats)

    def set_graphs(self, enable: bool):
        _check(lib().flip_batch_set_graphs(self.b, int(bool(enable))))

    def set_fused(self, enable: bool):
        """One launch per step kernel across all scenes, or per-scene launches (default)."""
        _check(lib().flip_batch_set_fused(self.b, int(bool(enable))))

    def form(self):
        """(fused, graphs): the form the batch's steps take."""
        f, g = C.c_int32(0), C.c_int32(0)
        _check(lib().flip_batch_get_form(self.b, C.byref(f), C.byref(g)))
        return bool(f.value), bool(g.value)

    def graph_active(self) -> bool:
        return bool(lib().flip_batch_graph_active(self.b))

    def set_team_exponent(self, exponent: float):
        _check(lib().flip_batch_set_team_exponent(self.b, float(exponent)))

    def autotune(self, sims, steps_per_candidate: int = 1) -> float:
        """Chooses the solve-team split by timing real steps (the scenes advance)."""
        hs = [s.h for s in sims]
        arr = (C.c_void_p * max(len(hs), 1))(*[h.value if isinstance(h, C.c_void_p) else h
                                                for h in hs])
        out = C.c_double(0.0)
        _check(lib().flip_batch_autotune(self.b, arr, len(hs), int(steps_per_candidate),
                                         C.byref(out)))
        return float(out.value)

    def close(self):
        if getattr(self, "b", None):
            flip_batch_destroy(self.b)
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def flip_footprint_bytes(params: FlipParams, np_: int) -> int:
    return int(lib().flip_footprint_bytes(C.byref(params), int(np_)))


class Server:
    """Continuous-batching step server (include/flip_server.h)."""

    def __init__(self, budget_bytes: int, max_batch: int):
        self.s = C.c_void_p()
        _check(lib().flip_server_create(int(budget_bytes), int(max_batch), C.byref(self.s)))

    def add_scene(self, params: FlipParams, x, y, z, u, v, w) -> int:
        bufs = [_buf(np.ascontiguousarray(a, np.float32), np.float32) for a in (x, y, z, u, v, w)]
        sid = C.c_int32(-1)
        _check(lib().flip_server_add_scene(self.s, C.byref(params),
                                           *[C.c_void_p(b[0]) for b in bufs], bufs[0][1] // 4,
                                           C.byref(sid)))
        return sid.value

    def submit(self, scene: int, t_arrival: float = -1.0) -> int:
        t = C.c_int64(-1)
        _check(lib().flip_server_submit(self.s, int(scene), float(t_arrival), C.byref(t)))
        return t.value

    def wait(self, ticket: int) -> RequestInfo:
        info = RequestInfo()
        _check(lib().flip_server_wait(self.s, int(ticket), C.byref(info)))
        return info

    def drain(self):
        _check(lib().flip_server_drain(self.s))

    def set_fused(self, enable: bool):
        """Fused batches, or per-scene launches inside each batch (default)."""
        _check(lib().flip_server_set_fused(self.s, int(bool(enable))))

    def set_overlap(self, enable: bool):
        """Overlapped batches (default) or one batch at a time."""
        _check(lib().flip_server_set_overlap(self.s, int(bool(enable))))

    def now(self) -> float:
        return float(lib().flip_server_now(self.s))

    def usage(self):
        r, b = C.c_int32(0), C.c_size_t(0)
        _check(lib().flip_server_usage(self.s, C.byref(r), C.byref(b)))
        return r.value, b.value

    def handle(self, scene: int):
        h = C.c_void_p()
        _check(lib().flip_server_scene_handle(self.s, int(scene), C.byref(h)))
        return h

    def particles(self, scene: int):
        """A resident scene's particles in creation order (call when it is idle)."""
        h = self.handle(scene)
        arrs = [flip_read(h, f) for f in (PX, PY, PZ, PU, PV, PW)]
        ids = flip_read(h, PID)
        inv = np.empty_like(ids)
        inv[ids] = np.arange(ids.size, dtype=ids.dtype)
        return [a[inv] for a in arrs]

    def remove_scene(self, scene: int):
        _check(lib().flip_server_remove_scene(self.s, int(scene)))

    def close(self):
        if getattr(self, "s", None):
            lib().flip_server_destroy(self.s)
            self.s = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def surface_default_params(params: FlipParams) -> FlipSurfaceParams:
    sp = FlipSurfaceParams()
    lib().flip_surface_default_params(C.byref(params), C.byref(sp))
    return sp


def surface_case_table():
    """(ntri[256], tri[256, 12, 3]) local-edge triangles of the library's case table."""
    ntri = np.zeros(256, np.uint8)
    tri = np.zeros((256, SURF_MAX_TRI, 3), np.uint8)
    _check(lib().flip_surface_case_table(ntri.ctypes.data, tri.ctypes.data))
    return ntri, tri


class Surface:
    """Surface reconstruction (Sec. 3.3) on a sampling grid: scalar field, marching
    cubes, vertex normals.  Owns a flip_surface object."""

    def __init__(self, sp: FlipSurfaceParams, stream=None):
        self.params = sp
        self.n = tuple(int(sp.n[a]) for a in range(3))
        out = C.c_void_p()
        _check(lib().flip_surface_create(C.byref(sp), stream, C.byref(out)))
        self.h = out
        self.nv = self.nt = 0

    def sdf(self, sim):
        _check(lib().flip_surface_sdf(self.h, sim.h if hasattr(sim, "h") else sim))

    def set_field(self, phi):
        a = np.ascontiguousarray(phi, dtype=np.float32)
        assert a.size == (self.n[0] + 1) * (self.n[1] + 1) * (self.n[2] + 1)
        _check(lib().flip_surface_set_field(self.h, a.ctypes.data, 0))

    def mesh(self):
        nv, nt = C.c_int64(0), C.c_int64(0)
        _check(lib().flip_surface_mesh(self.h, C.byref(nv), C.byref(nt)))
        self.nv, self.nt = nv.value, nt.value
        return self.nv, self.nt

    def read(self, which: int):
        shapes = {SURF_FIELD: ((self.n[2] + 1, self.n[1] + 1, self.n[0] + 1), np.float32),
                  SURF_VERTICES: ((self.nv, 3), np.float32), SURF_NORMALS: ((self.nv, 3), np.float32),
                  SURF_TRIANGLES: ((self.nt, 3), np.int32), SURF_VERTEX_EDGE: ((self.nv,), np.int64)}
        shape, dt = shapes[which]
        out = np.empty(shape, dt)
        _check(lib().flip_surface_read(self.h, which, out.ctypes.data, out.nbytes, 0))
        return out

    def close(self):
        if getattr(self, "h", None):
            lib().flip_surface_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Simulation:
    """One scene on the GPU: owns the handle and (by default) a torch CUDA stream."""

    def __init__(self, params: FlipParams, x, y, z, u, v, w, stream=None, allocator="torch"):
        import torch
        self._stream_obj = None
        if stream is None and torch.cuda.is_available():
            self._stream_obj = torch.cuda.Stream()
            stream = self._stream_obj.cuda_stream
        self.stream = stream
        self.params = params
        self.h, self._keep = flip_create(params, x, y, z, u, v, w, stream=stream,
                                         allocator=allocator)

    def step(self, nsteps: int = 1, stats: bool = False):
        return flip_step(self.h, nsteps, stats)

    def sync(self) -> int:
        return flip_sync(self.h)

    def read(self, field: int, out=None):
        return flip_read(self.h, field, out)

    def write(self, field: int, src):
        flip_write(self.h, field, src)

    def step_times(self):
        """Device ms of each step of the last step(..., stats=True) call (numpy)."""
        n = int(lib().flip_step_times(self.h, None, 0))
        if n < 0:
            _check(-n)
        out = np.zeros(n, np.float64)
        if n:
            lib().flip_step_times(self.h, out.ctypes.data_as(C.c_void_p), n)
        return out

    def set_wait_timeout(self, ns: int):
        """Limit of the handle's bounded device-side waits (0: the defaults)."""
        _check(lib().flip_set_wait_timeout(self.h, int(ns)))

    def set_solver_blocks(self, nblocks: int):
        _check(lib().flip_set_solver_blocks(self.h, int(nblocks)))

    def autotune_solver(self, steps_per_candidate: int = 1) -> int:
        """Chooses the solve's CTA count by timing real steps (the scene advances)."""
        out = C.c_int32(0)
        _check(lib().flip_autotune_solver(self.h, int(steps_per_candidate), C.byref(out)))
        return int(out.value)

    def set_transfer_ctas(self, p2g_per_sm: int, g2p_per_sm: int):
        """CTAs per SM of the P2G and G2P launches (0: the defaults)."""
        _check(lib().flip_set_transfer_ctas(self.h, int(p2g_per_sm), int(g2p_per_sm)))

    def transfer_ctas(self):
        """(P2G, G2P) CTAs per SM in use."""
        p, g = C.c_int32(0), C.c_int32(0)
        _check(lib().flip_get_transfer_ctas(self.h, C.byref(p), C.byref(g)))
        return int(p.value), int(g.value)

    def autotune_transfers(self, steps_per_candidate: int = 1):
        """Chooses the P2G and G2P launch shapes by timing real steps (the scene
        advances by 6 * steps_per_candidate steps); returns (P2G, G2P) CTAs per SM."""
        p, g = C.c_int32(0), C.c_int32(0)
        _check(lib().flip_autotune_transfers(self.h, int(steps_per_candidate), C.byref(p),
                                             C.byref(g)))
        return int(p.value), int(g.value)

    def energy(self, particle_mass: float):
        """(kinetic, potential, total) energy of the particles (Sec. 4, Fig. 10)."""
        return flip_energy(self.h, particle_mass)

    def particles(self, by_id: bool = True):
        """(x, y, z, u, v, w) as float32 numpy arrays, in creation order when by_id."""
        arrs = [self.read(f) for f in (PX, PY, PZ, PU, PV, PW)]
        if by_id:
            ids = self.read(PID)
            inv = np.empty_like(ids)
            inv[ids] = np.arange(ids.size, dtype=ids.dtype)
            arrs = [a[inv] for a in arrs]
        return arrs

    def close(self):
        if getattr(self, "h", None):
            flip_destroy(self.h)
            self.h = None
            self._keep = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
