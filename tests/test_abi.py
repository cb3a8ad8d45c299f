"""The C-ABI library builds, loads and exports every function include/flip.h declares;
host-side argument checks work without a GPU (no compute calls here)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def F():
    from paper_2404_01931_gb300 import build_lib
    build_lib.build()
    from paper_2404_01931_gb300 import flip
    flip.lib()
    return flip


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(flip_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for fn in ("flip_create", "flip_step", "flip_read", "flip_write", "flip_destroy",
               "flip_strerror", "flip_solve_pressure", "flip_sync"):
        assert fn in names


def test_every_declared_symbol_is_exported(F):
    lib = ctypes.CDLL(F.LIB_PATH)
    missing = [n for n in sorted(declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing


def test_abi_version_and_strerror(F):
    L = F.lib()
    assert L.flip_abi_version() == 5
    for code in range(9):
        assert L.flip_strerror(code).decode() != "unknown status"
    assert L.flip_strerror(99).decode() == "unknown status"


def test_struct_layouts_match_header(F):
    # flip_params: 3 int32 (+4) + 10 double + 7 int32 (+4) + cfl + 2 int32 + 2 int64
    assert ctypes.sizeof(F.FlipParams) == 12 + 4 + 10 * 8 + 28 + 4 + 8 + 8 + 16
    assert ctypes.sizeof(F.FlipStats) == 5 * 8 + 2 * 4 + 10 * 8 + 2 * 8
    # flip_surface_params: 3 int32 (+4 padding) + 7 double
    assert ctypes.sizeof(F.FlipSurfaceParams) == 12 + 4 + 7 * 8


def test_surface_default_params(F):
    p = F.default_params(40, 24, 32)
    sp = F.surface_default_params(p)
    assert list(sp.n) == [40, 24, 32] and list(sp.origin) == [0.0, 0.0, 0.0]
    assert sp.h == p.dx and sp.radius == 0.5 * p.dx and sp.search_radius == 2 * p.dx
    assert sp.iso == 0.0


def test_default_params(F):
    p = F.default_params(64, 32, 48)
    assert list(p.n) == [64, 32, 48] and p.dx == 1 / 64 and p.dt == 1 / 240
    assert p.gravity[1] == -9.81 and p.flip_ratio == 0.95 and p.cg_max_iter == 20 * 64
    assert p.skin == pytest.approx(1e-3 / 64)
    assert p.preconditioner == F.FLIP_PRECOND_MG and p.mg_smooth == 2 and p.warm_start == 0
    assert p.cfl == 0.0 and p.ppc_min == 0 and p.ppc_max == 0 and p.max_particles == 0


@pytest.mark.parametrize("field,value,code", [
    ("dx", 0.3, 1), ("dt", 0.0, 1), ("flip_ratio", 1.5, 1), ("skin", 0.0, 1),
    ("precision", 7, 1), ("cg_max_iter", 0, 1), ("rho", -1.0, 1), ("preconditioner", 5, 1),
    ("mg_smooth", 0, 1), ("warm_start", 2, 1), ("cfl", -1.0, 1), ("cfl", float("inf"), 1),
    ("ppc_min", 65, 1), ("ppc_max", -1, 1), ("max_particles", -5, 1)])
def test_argument_checks_before_any_device_call(F, field, value, code):
    p = F.default_params(16)
    setattr(p, field, value)
    x = np.zeros(4, np.float32)
    with pytest.raises(F.FlipError) as ei:
        F.flip_create(p, x, x, x, x, x, x, allocator=None)
    assert ei.value.code == code


def test_grid_size_checks(F):
    p = F.default_params(16)
    p.n[0] = 1
    x = np.zeros(4, np.float32)
    with pytest.raises(F.FlipError):
        F.flip_create(p, x, x, x, x, x, x, allocator=None)


def test_largest_grid_edge(F):
    """Every face index must fit in 31 bits ((n+1)^3 < 2^31): 1289^3 passes the
    parameter checks (and then needs a device), 1290^3 is refused before any device
    call."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("host-only check (a GPU would allocate the grid)")
    x = np.zeros(4, np.float32)
    with pytest.raises(F.FlipError) as ei:
        F.flip_create(F.default_params(1290), x, x, x, x, x, x, allocator=None)
    assert ei.value.code == F.FLIP_E_ARG and "too large" in str(ei.value)
    with pytest.raises(F.FlipError) as ei:
        F.flip_create(F.default_params(1289), x, x, x, x, x, x, allocator=None)
    assert ei.value.code == F.FLIP_E_NOGPU


def test_mismatched_particle_arrays(F):
    p = F.default_params(16)
    with pytest.raises(ValueError):
        F.flip_create(p, *[np.zeros(4, np.float32)] * 5, np.zeros(5, np.float32),
                      allocator=None)


def test_wrong_dtype_rejected(F):
    p = F.default_params(16)
    with pytest.raises(TypeError):
        F.flip_create(p, *[np.zeros(4, np.float64)] * 6, allocator=None)


def test_server_and_batch_need_a_gpu(F):
    import torch
    if torch.cuda.is_available():
        pytest.skip("host-only check")
    with pytest.raises(F.FlipError) as ei:
        F.Server(1 << 30, 4)
    assert ei.value.code == F.FLIP_E_NOGPU
    with pytest.raises(F.FlipError) as ei:
        F.flip_batch_create(4)
    assert ei.value.code == F.FLIP_E_NOGPU
    assert F.flip_footprint_bytes(F.default_params(16), 100) == 0  # no device to size for


@pytest.mark.parametrize("n", [48, 49, 57, 83, 97, 191])
def test_default_params_are_valid_for_every_edge(F, n):
    """1/(1/n) is not always n in FP64; the defaults must still pass the checks (the
    create call then succeeds on a GPU and fails only for want of one elsewhere)."""
    p = F.default_params(n)
    x = np.full(4, 0.5, np.float32)
    try:
        h, _keep = F.flip_create(p, x, x, x, np.zeros(4, np.float32), np.zeros(4, np.float32),
                                 np.zeros(4, np.float32), allocator=None)
    except F.FlipError as e:
        assert e.code == F.FLIP_E_NOGPU
    else:
        F.flip_destroy(h)


def test_no_library_no_fallback():
    """Without the shared library every entry point raises: there is no CPU path."""
    import subprocess
    import sys
    code = (
        "import numpy as np\n"
        "from paper_2404_01931_gb300 import flip as F\n"
        "F.LIB_PATH = '/nonexistent/libflip_gb300.so'\n"
        "x = np.zeros(4, np.float32)\n"
        "for call in (lambda: F.lib(), lambda: F.default_params(16),\n"
        "             lambda: F.flip_create(F.FlipParams(), x, x, x, x, x, x, allocator=None)):\n"
        "    try:\n"
        "        call()\n"
        "    except RuntimeError as e:\n"
        "        assert 'not built' in str(e), e\n"
        "    else:\n"
        "        raise SystemExit('an entry point ran without the library')\n"
        "print('ok')\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr


def test_headers_compile_as_c_and_link(F, tmp_path):
    """include/*.h are plain C (C11, -Wall -Werror) and a C program links against the
    library and calls its host-only entry points (no device needed)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "abi_check.c"
    src.write_text(
        '#include "flip.h"\n#include "flip_server.h"\n#include "flip_surface.h"\n'
        "#include <stdio.h>\n"
        "int main(void) {\n"
        "  flip_params p;\n"
        "  flip_default_params(&p, 32, 32, 32);\n"
        "  if (flip_abi_version() != FLIP_ABI_VERSION) return 1;\n"
        "  if (p.n[0] != 32 || !(p.dx > 0.0)) return 2;\n"
        "  if (flip_strerror(FLIP_E_ARG) == NULL) return 3;\n"
        "  printf(\"ok %d\\n\", flip_abi_version());\n"
        "  return 0;\n"
        "}\n")
    exe = tmp_path / "abi_check"
    libdir = os.path.dirname(F.LIB_PATH)
    r = subprocess.run([cc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-I",
                        os.path.join(ROOT, "include"), str(src), "-o", str(exe), "-L", libdir,
                        "-lflip_gb300", f"-Wl,-rpath,{libdir}"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.startswith("ok "), (r.returncode, r.stdout, r.stderr)


def test_surface_bin_grid_limit(F):
    """The particle bins of the surface object are indexed in 32 bits: a search radius
    too small for the sampling grid is refused before any device call; the defaults
    at the largest grid pass the checks."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("host-only check (a GPU would allocate the bins)")
    sp = F.surface_default_params(F.default_params(1024))
    sp.search_radius, sp.radius = sp.h, 0.25 * sp.h        # 2053^3 bins
    with pytest.raises(F.FlipError) as ei:
        F.Surface(sp)
    assert ei.value.code == F.FLIP_E_ARG and "bin grid" in str(ei.value)
    with pytest.raises(F.FlipError) as ei:
        F.Surface(F.surface_default_params(F.default_params(1024)))   # 1029^3 bins
    assert ei.value.code == F.FLIP_E_NOGPU


def test_solve_wrappers_check_buffer_sizes(F):
    """The standalone solves read and write one entry per cell of params.n: a short
    buffer is refused on the host before any device call."""
    import torch
    p = F.default_params(8)
    nc = 8 ** 3
    t = torch.zeros(nc, dtype=torch.uint8)
    good = torch.zeros(nc, dtype=torch.float32)
    short = torch.zeros(nc - 1, dtype=torch.float32)
    for fn in (F.flip_solve_pressure, F.flip_solve_pressure_noalloc):
        for args in ((t, short, good), (t, good, short), (t[:-1], good, good)):
            with pytest.raises(F.FlipError) as ei:
                fn(p, *args)
            assert ei.value.code == F.FLIP_E_SIZE


@pytest.mark.parametrize("field,value", [("dx", 0.3), ("dt", float("inf")), ("dx", 0.0),
                                         ("rho", -1.0), ("cg_max_iter", 0),
                                         ("precision", 1)])
def test_both_solves_refuse_the_same_params(F, field, value):
    """flip_solve_pressure and its allocation-free variant share their parameter
    checks: both refuse (FLIP_E_ARG) before touching a device."""
    p = F.default_params(8)
    setattr(p, field, value)
    L = F.lib()
    it = ctypes.c_int32(0)
    rel = ctypes.c_double(0.0)
    args = (ctypes.byref(p), None, None, None, None, ctypes.byref(it), ctypes.byref(rel))
    assert L.flip_solve_pressure(*args) == F.FLIP_E_ARG
    assert L.flip_solve_pressure_noalloc(*args) == F.FLIP_E_ARG


def test_precision_entry_points_check_arguments(F):
    """flip_dot_f32 and flip_residual_pairs refuse bad arguments on the host."""
    L = F.lib()
    out = ctypes.c_double(0.0)
    assert L.flip_dot_f32(None, None, -1, ctypes.byref(out), None) == F.FLIP_E_ARG
    assert L.flip_dot_f32(None, None, 4, None, None) == F.FLIP_E_ARG
    assert L.flip_dot_f32(None, None, 4, ctypes.byref(out), None) == F.FLIP_E_ARG
    p = F.default_params(8)
    p.dx = 0.3
    assert L.flip_residual_pairs(ctypes.byref(p), *([None] * 7), None) == F.FLIP_E_ARG
    p = F.default_params(8)
    assert L.flip_residual_pairs(ctypes.byref(p), *([None] * 7), None) == F.FLIP_E_ARG
    import torch
    with pytest.raises(F.FlipError) as ei:
        F.flip_dot_f32(torch.zeros(4), torch.zeros(5))
    assert ei.value.code == F.FLIP_E_SIZE


def test_handle_entry_points_refuse_null(F):
    L = F.lib()
    assert L.flip_step_times(None, None, 0) == -F.FLIP_E_ARG
    assert L.flip_set_wait_timeout(None, 1000) == F.FLIP_E_ARG


def test_solve_trace_variant_compiles(tmp_path):
    """The solver's trace hooks (-DFLIP_SOLVE_TRACE) compile, and the trace entry
    point exists only in that variant (the normal build compiles the hooks out)."""
    import subprocess
    from paper_2404_01931_gb300 import build_lib
    src = os.path.join(build_lib.CSRC, "k_mg.cu")
    for trace in (True, False):
        obj = str(tmp_path / f"k_mg_{int(trace)}.o")
        cmd = [build_lib.nvcc(), *build_lib._flags(["-DFLIP_SOLVE_TRACE"] if trace else []),
               "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr[-2000:]
        nm = subprocess.run(["nm", "-g", obj], capture_output=True, text=True).stdout
        assert ("flip_solve_trace" in nm) == trace
