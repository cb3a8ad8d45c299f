"""Per-phase times of the multigrid-preconditioned solve, from the solve-trace build.

    python -m paper_2404_01931_gb300.solve_trace [--n 256] [--scene pool|dam]
                                                [--precision mixed|fp32] [--reps 3]

Builds the library with -DFLIP_SOLVE_TRACE into _lib_trace/ (the normal build is
untouched), steps a seeded scene, and after each traced step prints the phases of
its solve: the set-up (level flags, active-segment lists, codes, CTA-local lists,
start pass), the first three CG iterations (V-cycle, phase A, phase B), the end,
and the pieces of the last V-cycle by level.  Each time is the global-timer
difference between stamps that the first CTA takes after the grid barrier ending
a phase, so it includes that barrier.
"""
from __future__ import annotations

import argparse
import ctypes as C

import numpy as np

from . import build_lib

# slots of the kernel's trace (TraceSlot in csrc/k_mg.cu)
SETUP = [(0, "kernel entry"), (1, "shared tables"), (2, "block flags cleared")] + [
    (2 + l, f"fluid flags, level {l}") for l in range(1, 12)] + [
    (14, "active segments counted"), (15, "active-segment lists"), (16, "neighbour codes"),
    (17, "segment cache"), (18, "CTA-local lists (first CTA)"), (19, "start pass")]
ITER = [(20 + 3 * i + k, f"iteration {i + 1}: {name}") for i in range(3)
        for k, name in enumerate(("V-cycle", "phase A", "phase B"))]
END = [(29, "rest of the CG loop"), (30, "end pass"), (31, "kernel exit")]
VCYCLE = {32: "level 0: first black half-sweep", 33: "level 0: rest of pre-smoothing",
          34: "restriction 0 -> 1", 46: "CTA-local levels", 58: "level 0: correction + black",
          59: "level 0: post-smoothing but the last red"}
VCYCLE.update({34 + l: f"level {l}: down" for l in range(1, 12)})
VCYCLE.update({46 + l: f"level {l}: up" for l in range(1, 12)})
REFINE = [(60, "first refinement: entered"), (61, "first refinement: x += d"),
          (62, "first refinement: residual b - A x")]


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--scene", choices=("pool", "dam"), default="pool")
    ap.add_argument("--precision", choices=("mixed", "fp32"), default="mixed")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=2)
    args = ap.parse_args(argv)

    from . import flip as F
    from . import scenes as S
    F.LIB_PATH = build_lib.build(trace=True)
    lib = F.lib()
    lib.flip_solve_trace.argtypes = [C.POINTER(C.c_ulonglong), C.c_int]
    sc = S.pool_drop(args.n) if args.scene == "pool" else S.dam_break(args.n, 0.45, 0.5, seed=0)
    p = F.default_params(args.n)
    if args.precision == "mixed":
        p.precision = F.FLIP_PREC_MIXED_IR
        p.cg_tol, p.ir_tol = 1e-3, 1e-8
    print(f"# solve trace: {args.scene} {args.n}^3, {sc.n_particles} particles, {args.precision}")
    with F.Simulation(p, *sc.arrays()) as sim:
        sim.step(args.warmup)
        for rep in range(args.reps):
            rc, st = sim.step(1, stats=True)
            buf = (C.c_ulonglong * 64)()
            if lib.flip_solve_trace(buf, 64) != 0:
                raise RuntimeError("flip_solve_trace failed")
            t = np.array(list(buf), dtype=np.int64)
            t0 = t[0]
            print(f"\n## step {rep + 1}: solve {st.ms_pcg:.3f} ms (CUDA events), "
                  f"{st.cg_iterations} CG iterations, {st.ir_iterations} refinements\n")
            print("| phase | µs | since entry, µs |\n|---|---|---|")
            prev = t0
            for slot, name in SETUP + ITER + END:
                if t[slot] >= t0 > 0:  # stamped during this solve
                    print(f"| {name} | {(t[slot] - prev) / 1e3:.1f} | {(t[slot] - t0) / 1e3:.1f} |")
                    prev = t[slot]
            if all(t[s] >= t0 > 0 for s, _ in REFINE):
                print("\n| first refinement (mixed precision) | µs |\n|---|---|")
                for (a, _), (b, name) in zip(REFINE, REFINE[1:]):
                    print(f"| {name.split(': ')[1]} | {(t[b] - t[a]) / 1e3:.1f} |")
            pieces = sorted((s for s in VCYCLE if t[s] >= t0 > 0), key=lambda s: t[s])
            if pieces:
                print("\n| last V-cycle: piece | µs |\n|---|---|")
                for a, b in zip(pieces, pieces[1:]):
                    print(f"| {VCYCLE[b]} | {(t[b] - t[a]) / 1e3:.1f} |")


if __name__ == "__main__":
    main()
