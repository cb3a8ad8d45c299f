"""FLIP step benchmark: particle-steps/s on one GB300 (or N replicas), one JSON line.

Default workload: the drop-into-pool scene on a 256^3 MAC grid (pool depth 0.3 plus a
sphere of radius 0.15 at (0.5, 0.7, 0.5), 8 particles per fluid cell, 42,266,944
particles), mixed precision (FP32 multigrid-preconditioned CG on a correction that is
folded into a float-pair (~48-bit) solution, with the residual recomputed in float pairs,
to a relative residual of 1e-8; FP64 right-hand side and result), dt = 1/240, FLIP
ratio 0.95, seed 0.  Inputs are synthetic (seeded jittered seeding), generated on the
host.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload pool256|dam128|dam32]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores

A "step" is one full FLIP step (bin, P2G, divergence, PCG, G2P).  Timing: W untimed
steps, then K steps between CUDA events on the simulation's stream, bracketed by a
barrier and a synchronize; the max over ranks is reported.  The library records CUDA
events around every step and stage inside the timed call (read once after it), which
give the per-step latency percentiles and the per-stage rooflines.  The particle and
grid arrays (> 1 GB) are larger than the 129 MB L2, so no flush is needed between steps.
Outside the timed region, the first step of the seeded scene is compared field by field
with the FP64 oracle's (error_vs_oracle).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "pool256": dict(desc="drop into pool, 256^3, depth 0.3 + sphere r=0.15 at (0.5,0.7,0.5)",
                    n=256, scene="pool", precision="mixed", cg_tol=1e-3, ir_tol=1e-8),
    "pool128": dict(desc="drop into pool, 128^3, depth 0.3 + sphere r=0.15 at (0.5,0.7,0.5)",
                    n=128, scene="pool", precision="mixed", cg_tol=1e-3, ir_tol=1e-8),
    "dam128": dict(desc="dam break, 128^3, block x<0.25 y<0.5", n=128, scene="dam",
                   precision="fp32", cg_tol=1e-6, ir_tol=1e-8),
    "dam32": dict(desc="dam break, 32^3, block x<0.25 y<0.5", n=32, scene="dam",
                  precision="fp32", cg_tol=1e-6, ir_tol=1e-8),
    "dam64": dict(desc="dam break, 64^3, block x<0.25 y<0.5", n=64, scene="dam",
                  precision="fp32", cg_tol=1e-6, ir_tol=1e-8),
    "ddam128": dict(desc="double dam break, 128^3, blocks x<0.2 and x>0.8, y<0.5", n=128,
                    scene="ddam", precision="fp32", cg_tol=1e-6, ir_tol=1e-8),
    "drop128": dict(desc="water drop, 128^3, sphere r=0.2 at (0.5,0.6,0.5)", n=128,
                    scene="drop", precision="fp32", cg_tol=1e-6, ir_tol=1e-8),
    "drop104": dict(desc="water drop, 104^3, sphere r=0.2 at (0.5,0.6,0.5)", n=104,
                    scene="drop", precision="fp32", cg_tol=1e-6, ir_tol=1e-8),
}

# With the multigrid preconditioner, per fluid cell of level 0 and iteration
# (colour-split FP32 vectors, 16-bit neighbour codes):
#   phase A: read z, p_old, code (10 B); write p_new, q (8 B)        = 18 B
#   phase B: read d, p_new, q, r, code (18 B); write d, r, half of z = 26 B
#   V-cycle at level 0 with nu = 2: seven half-sweeps, each reading r, code and
#   the other colour's z and writing its colour's z for half the cells (~5 B),
#   the restriction reading r, z, code of the red cells (~5 B); coarser levels
#   add about a seventh of level 0's cycle                         ~ 92 B in all
#   refinement (float pairs): x += d (read x, d, write x, d: 24 B),
#   r = b - A x (read x, b, code, write r, half of z: 23 B)       => 47 B
#   per solve: b as a float pair from b64 (16 B), the solution out (x64, pff: 24 B)
MG_PCG_BYTES_PER_ITER = 92
MG_IR_BYTES_PER_OUTER = 47
MG_IR_BYTES_PER_SOLVE = 40
# The method-level byte model of a Jacobi-style PCG iteration per fluid cell
# (SpMV + dot 9 B, axpy + preconditioner + dot 25 B, p update 13 B) and of one
# outer refinement of the mixed mode (the solution read and written at 8 B each,
# the right-hand side read at 8 B, the residual written, neighbour reads: ~40 B):
# the algorithmic bytes of `roofline`.  The preconditioner's own passes (the
# V-cycle) are not algorithmic bytes of the method; the builder's model above
# counts them and is reported beside it.
METHOD_PCG_BYTES_PER_ITER = 47
METHOD_IR_BYTES_PER_OUTER = 40
# DRAM traffic of one k_pcg_mg launch on the 256^3 pool, read from the committed
# single-pass ncu summary, which records the hash of the solver's sources it was
# measured on; when the sources have changed since, the traffic is reported as null.
PCG_PROFILE = os.path.join(ROOT, "profiles", "k_pcg_mg_pool256_dram.md")
SOLVER_SOURCES = ("k_mg.cu", "pcg_common.cuh", "flip_kernels.cuh", "flip_internal.cuh")
# GB300's nominal HBM3e bandwidth, reported beside the measured copy bandwidth
NOMINAL_HBM_GBS = 7900.0


def solver_source_hash():
    """SHA-256 (first 16 hex digits) of the sources the persistent solve is built from."""
    h = hashlib.sha256()
    for name in SOLVER_SOURCES:
        with open(os.path.join(ROOT, "paper_2404_01931_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_pcg_traffic():
    """(bytes per launch, note): the DRAM traffic of the committed capture, when it was
    taken on the current solver sources; else (None, why)."""
    try:
        text = open(PCG_PROFILE).read()
    except OSError:
        return None, "no committed capture"
    vals = dict(re.findall(r"^(source_hash|dram_bytes_per_launch):\s*(\S+)", text, re.M))
    if "source_hash" not in vals or "dram_bytes_per_launch" not in vals:
        return None, "capture carries no source hash"
    if vals["source_hash"] != solver_source_hash():
        return None, (f"stale: captured on solver sources {vals['source_hash']}, "
                      f"now {solver_source_hash()}")
    return float(vals["dram_bytes_per_launch"]), f"ncu capture on sources {vals['source_hash']}"


def stage_roofline(w, np_, nfl, stage_ms, steps, peak):
    """Achieved HBM GB/s of the other stages over the live CUDA-event stage time, against
    the measured copy bandwidth, by two byte models.
    The method's algorithmic bytes (`frac`):
      bin:        56 B per particle (24 B read, key 4 B, 24 B written, histogram 4 B)
                  + 8 B per cell
      P2G:        24 B per particle + 21 B per cell (u*, v*, w* written 12 B, type 1 B,
                  start/count 8 B)
      divergence: 13 B per fluid cell
      G2P:        48 B per particle + 17 B per cell
    This build's traffic model (`frac_builder_model`):
      bin:        scatter 64 B per particle (key, rank, 28 B read, 28 B write) +
                  13 B per key (count read and clear, local start, cell type)
      P2G:        24 B per particle (positions and velocities, read once) +
                  20 B per face (accumulator read and clear, u_old write)
      divergence: 41 B per cell (type, 3 faces, b in FP64, solution zeroed)
      G2P:        56 B per particle (24 B in, 24 B out, key and rank)"""
    n = w["n"]
    cells = n ** 3
    keys = (-(-n // 8) * 8) ** 3
    faces = 3 * (n + 1) * n * n
    method = {"bin": 56 * np_ + 8 * cells, "p2g": 24 * np_ + 21 * cells,
              "divergence": 13 * nfl, "g2p": 48 * np_ + 17 * cells}
    builder = {"bin": 64 * np_ + 13 * keys, "p2g": 24 * np_ + 20 * faces,
               "divergence": 41 * cells, "g2p": 56 * np_}
    out = {}
    for k in method:
        t = stage_ms[k] / steps / 1e3
        gbs = method[k] / t / 1e9 if t > 0 else None
        gbs_b = builder[k] / t / 1e9 if t > 0 else None
        out[k] = {"achieved_gbs": gbs, "frac": gbs / peak if gbs else None,
                  "frac_of_nominal": gbs / NOMINAL_HBM_GBS if gbs else None,
                  "algorithmic_bytes": method[k],
                  "frac_builder_model": gbs_b / peak if gbs_b else None,
                  "builder_model_bytes": builder[k]}
    return out


def make_scene(w, n=None):
    """The workload's scene at its grid edge (or at edge n)."""
    from paper_2404_01931_gb300 import scenes as S
    n = w["n"] if n is None else n
    if w["scene"] == "pool":
        return S.pool_drop(n)
    if w["scene"] == "ddam":
        return S.double_dam_break(n)
    if w["scene"] == "drop":
        return S.water_drop(n)
    return S.dam_break(n)


def make_params(w):
    from paper_2404_01931_gb300 import flip as F
    p = F.default_params(w["n"])
    p.cg_tol = w["cg_tol"]
    p.ir_tol = w["ir_tol"]
    if w["precision"] == "mixed":
        p.precision = F.FLIP_PREC_MIXED_IR
    return p


L2_BYTES = 126 << 20  # GB300 L2 (129 MB nominal, 126 MiB as reported)


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self._t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "50"], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self._t:
            self._t.join(timeout=2)
        return self.summarize(self.lines)

    @staticmethod
    def summarize(lines):
        """Median SM clock under load, the maximum clock and every throttle reason
        seen active, from nvidia-smi's noheader/nounits CSV lines (FIELDS order)."""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _reduce(x, ws, op):
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda") if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x, ws):
    """The largest value over the ranks (the job's time is the slowest rank's)."""
    import torch.distributed as dist
    return _reduce(x, ws, dist.ReduceOp.MAX if ws > 1 else None)


def sum_over_ranks(x, ws):
    import torch.distributed as dist
    return _reduce(x, ws, dist.ReduceOp.SUM if ws > 1 else None)


def job_rate(units, seconds, ws):
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return sum_over_ranks(units, ws) / max_over_ranks(seconds, ws)


def shard_scenes(weights, n_ranks):
    """Host-side router of independent scenes over ranks (one GPU each): longest
    processing time first, each scene to the least-loaded rank (ties: the lower rank).
    Deterministic, so every rank computes the same plan with no communication.
    Returns each rank's scene indices in ascending order."""
    load = [0.0] * n_ranks
    out = [[] for _ in range(n_ranks)]
    for i in sorted(range(len(weights)), key=lambda i: (-weights[i], i)):
        r = min(range(n_ranks), key=lambda r: (load[r], r))
        out[r].append(i)
        load[r] += weights[i]
    return [sorted(o) for o in out]


def _rel_l2(a, b, floor=0.0):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), floor, 1e-300))


def first_step_fields(sim, F):
    """Fields of a handle right after its first step: faces, pressure, right-hand side
    and the particles in creation order."""
    return {"u_old": [sim.read(f) for f in (F.U_OLD, F.V_OLD, F.W_OLD)],
            "u_new": [sim.read(f) for f in (F.U_NEW, F.V_NEW, F.W_NEW)],
            "p": sim.read(F.PRESSURE_F64), "rhs": sim.read(F.RHS),
            "type": sim.read(F.CELL_TYPE), "particles": sim.particles()}


def error_vs_oracle(w, sc, got):
    """Per-field error of the GPU's first step of the seeded scene against the FP64
    oracle's step from the same input, on the host, outside the timed region.  Mixed
    mode is compared with a tight oracle solve (CG to 1e-11), FP32 mode with the
    oracle's same solver and tolerance.  Velocity norms are floored at g dt sqrt(n)."""
    import oracle as O
    n = w["n"]
    mixed = w["precision"] == "mixed"
    op = O.Params(n=(n, n, n), dx=1.0 / n, cg_tol=1e-11 if mixed else w["cg_tol"],
                  cg_max_iter=100000 if mixed else 0)
    t0 = time.perf_counter()
    ref = O.step(op, *sc.arrays())
    el = time.perf_counter() - t0
    gdt = 9.81 / 240
    nf = (n + 1) * n * n
    fl = gdt * np.sqrt(3 * nf)
    x, y, z, u, v, wv = got["particles"]
    out = {
        "reference": "FP64 oracle step from the same seeded input, "
                     + ("tight solve (CG to 1e-11)" if mixed else
                        f"same multigrid-PCG to {w['cg_tol']:g}"),
        "oracle_s": round(el, 1), "oracle_cores": O.num_threads(),
        "cell_type_mismatches": int(np.count_nonzero(got["type"].ravel() != ref.type.ravel())),
        "u_old_rel_l2": _rel_l2(np.concatenate([a.ravel() for a in got["u_old"]]),
                                np.concatenate([a.ravel() for a in ref.u_old]), fl),
        "rhs_rel_l2": _rel_l2(got["rhs"], ref.rhs),
        "pressure_rel_l2": _rel_l2(got["p"], ref.pressure),
        "u_new_rel_l2": _rel_l2(np.concatenate([a.ravel() for a in got["u_new"]]),
                                np.concatenate([a.ravel() for a in ref.u_new]), fl),
        "position_max_err_cells": float(np.abs(np.stack([x, y, z]).astype(np.float64)
                                               - np.stack([ref.x, ref.y, ref.z])).max() * n),
        "velocity_rel_l2": _rel_l2(np.stack([u, v, wv]), np.stack([ref.u, ref.v, ref.w]),
                                   gdt * np.sqrt(3 * x.size)),
        "bar": "relative L2 <= 1e-5 for grid velocities and pressure; positions within "
               "1e-4 of a cell",
    }
    return out


def cpu_baseline(w, budget_s=25.0):
    """The FP64 oracle timed on this host's cores on a bounded sample of the workload."""
    import oracle as O
    from paper_2404_01931_gb300 import scenes as S
    n = w["n"]
    # Sample: the same scene shape at the largest grid edge whose oracle step fits the
    # budget (the full 256^3 step takes longer than the budget on typical hosts).
    for ns in ([n, n // 2, n // 4, 32] if n > 32 else [n]):
        sc = S.pool_drop(ns) if w["scene"] == "pool" else S.dam_break(ns)
        op = O.Params(n=(ns, ns, ns), dx=1.0 / ns, cg_tol=w["ir_tol"] if w["precision"] == "mixed"
                      else w["cg_tol"])
        t0 = time.perf_counter()
        r = O.step(op, *sc.arrays(), fields=False)
        dt = time.perf_counter() - t0
        if dt <= budget_s or ns == 32:
            steps = 1
            st = [r.x, r.y, r.z, r.u, r.v, r.w]
            while (time.perf_counter() - t0) + dt <= budget_s and steps < 10:
                r = O.step(op, *st, fields=False)
                st = [r.x, r.y, r.z, r.u, r.v, r.w]
                steps += 1
            el = time.perf_counter() - t0
            out = {"value": sc.n_particles * steps / el, "unit": "particle-steps/s",
                   "cores": O.num_threads(), "kind": "oracle",
                   "sample": f"{steps} oracle step(s) of the same scene at {ns}^3 "
                             f"({sc.n_particles} particles), FP64, {el:.1f} s"}
            out["single_thread"] = cpu_single_thread(w)
            return out
    return None


def cpu_single_thread(w):
    """The same oracle on one host thread: one step of the scene at 64^3 (or the
    workload's edge if smaller)."""
    import oracle as O
    from paper_2404_01931_gb300 import scenes as S
    ns = min(w["n"], 64)
    sc = S.pool_drop(ns) if w["scene"] == "pool" else S.dam_break(ns)
    op = O.Params(n=(ns, ns, ns), dx=1.0 / ns, cg_tol=w["ir_tol"] if w["precision"] == "mixed"
                  else w["cg_tol"])
    cores = O.num_threads()
    O.set_num_threads(1)
    try:
        t0 = time.perf_counter()
        O.step(op, *sc.arrays(), fields=False)
        el = time.perf_counter() - t0
    finally:
        O.set_num_threads(cores)
    return {"value": sc.n_particles / el, "unit": "particle-steps/s", "cores": 1,
            "sample": f"1 oracle step of the same scene at {ns}^3 ({sc.n_particles} "
                      f"particles), FP64, one thread, {el:.1f} s"}


def run_reference(args, w):
    ws, rank, _ = dist_setup()
    if rank != 0:
        return
    import oracle as O
    from paper_2404_01931_gb300 import scenes as S
    n = w["n"]
    # each step: one oracle step of the workload's scene, on the workload's own grid
    # when the K + W steps fit about three minutes of the host's cores (the oracle
    # takes ~6.6 s per step at 256^3 on 16 cores, ~0.09 s at 64^3, about in
    # proportion to the cells), else on the largest halved grid that does
    ns = n
    while ns > 16 and (args.steps + args.warmup) * 6.6 * (ns / 256.0) ** 3 > 180.0:
        ns //= 2
    sc = make_scene(w, ns)
    op = O.Params(n=(ns, ns, ns), dx=1.0 / ns,
                  cg_tol=w["ir_tol"] if w["precision"] == "mixed" else w["cg_tol"])
    st = [a.astype(np.float64) for a in sc.arrays()]
    for _ in range(args.warmup):
        r = O.step(op, *st, fields=False)
        st = [r.x, r.y, r.z, r.u, r.v, r.w]
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r = O.step(op, *st, fields=False)
        st = [r.x, r.y, r.z, r.u, r.v, r.w]
    el = time.perf_counter() - t0
    val = sc.n_particles * args.steps / el
    sample = f"oracle step of the same scene at {ns}^3 ({sc.n_particles} particles), FP64"
    out = {"metric": "FLIP particle-steps/s", "value": val, "unit": "particle-steps/s",
           "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": el * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": w["desc"], "grid": [n, n, n], "reference_sample_grid": ns},
           "cpu_baseline": {"value": val, "unit": "particle-steps/s", "cores": O.num_threads(),
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": val, "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def batch_stage_roofline(scenes, nfl_total, stage_ms, steps, peak):
    """The stage rooflines of a batch (the method's byte model, as stage_roofline),
    summed over its scenes, over the fused form's batch-wide stage times."""
    np_ = sum(sc.n_particles for sc in scenes)
    cells = sum(int(np.prod(sc.n)) for sc in scenes)
    model = {"bin": 56 * np_ + 8 * cells, "p2g": 24 * np_ + 21 * cells,
             "divergence": 13 * nfl_total, "g2p": 48 * np_ + 17 * cells}
    out = {}
    for k, b in model.items():
        t = stage_ms[k] / steps / 1e3
        gbs = b / t / 1e9 if t > 0 else None
        out[k] = {"achieved_gbs": gbs, "frac": gbs / peak if gbs else None,
                  "algorithmic_bytes": b, "ms_per_step": stage_ms[k] / steps}
    return out


def run_batch(args):
    """64 independent dam-break scenes, edges {32,48,64,80,96} and fluid fraction
    0.2-0.5 by seed, stepped together: the fused form (one launch per step kernel
    for all scenes, one batched solve launch), mixed precision unless --precision
    fp32.  Also times, on the same scenes: the fused form replayed as CUDA graphs,
    the per-scene-launch form, and one flip_step per scene after another."""
    import torch
    import torch.distributed as dist

    import __graft_entry__
    ws, rank, local = dist_setup()
    if rank == 0 or ws == 1:
        __graft_entry__.build()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist.barrier()
        __graft_entry__.build()
    from paper_2404_01931_gb300 import flip as F
    from paper_2404_01931_gb300 import scenes as S
    mixed = (args.precision or "mixed") == "mixed"
    every = S.batch_scenes(args.batch, seed=0)
    # N GPUs: the scenes are sharded by the router, with no data-path collective
    mine = shard_scenes([sc.n_particles for sc in every], ws)[rank]
    scenes = [every[i] for i in mine]
    sims = []
    for sc in scenes:
        p = F.default_params(sc.n[0])
        if mixed:
            p.precision = F.FLIP_PREC_MIXED_IR
            p.cg_tol, p.ir_tol = 1e-3, 1e-8
        sims.append(F.Simulation(p, *sc.arrays()))
    npart = sum(sc.n_particles for sc in scenes)
    footprint = sum(F.flip_footprint_bytes(sim.params, sc.n_particles)
                    for sim, sc in zip(sims, scenes))
    stream = torch.cuda.Stream()  # the batch's launches run here; it joins every scene
    b = F.Batch(len(sims), stream=stream.cuda_stream)
    b.set_fused(args.batch_fused)
    # warm-up, then the autotuner picks the solve-team split and the step's form
    # (fused or per-scene launches, stream-ordered or graph-replayed) on real steps
    if args.warmup:
        b.step(sims, args.warmup)
    exponent = b.autotune(sims, 1) if args.autotune else 1.0
    form = b.form()

    def timed(k):
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc_, _ = b.step(sims, k)
        e1.record(stream)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        return rc_, max_over_ranks(e0.elapsed_time(e1), ws)

    def form_name(fused, graphs):
        return ("fused" if fused else "per-scene launches") + (", graph replay" if graphs else "")

    # The scenes evolve as they step (a collapsing column spreads over more cells, so
    # later steps cost more): every timed form starts from the initial particles,
    # warmed by two steps.
    init = [sc.arrays() for sc in scenes]

    def restart():
        for sim, arr in zip(sims, init):
            ids = sim.read(F.PID)
            F.flip_write_particles(sim.h, *[np.ascontiguousarray(a[ids]) for a in arr])
        b.step(sims, 2)

    ksteps = args.steps - args.steps % 2  # graph replays run pairs of steps
    restart()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    rc, ms = timed(ksteps)
    ck = clocks.stop()
    units = sum_over_ranks(npart * ksteps, ws)
    # the other forms on the same scenes, from the same state
    forms = {}
    for fused, graphs in ((True, False), (True, True), (False, False), (False, True)):
        if (fused, graphs) == form:
            continue
        b.set_fused(fused)
        b.set_graphs(graphs)
        restart()
        _, t = timed(ksteps)
        forms[form_name(fused, graphs)] = {"ms_per_step": t / ksteps, "value": units / (t / 1e3)}
    # stage times (the fused form's batch-wide stages) and iteration counts from one
    # more step with statistics (untimed), from the same state
    b.set_graphs(form[1])
    b.set_fused(True)
    restart()
    rc_st, st = b.step(sims, 1, stats=True)
    b.set_fused(form[0])
    rc = rc or rc_st
    nfl = sum(x.n_fluid_cells for x in st)
    stage_ms = {"bin": st[0].ms_bin, "p2g": st[0].ms_p2g, "divergence": st[0].ms_divergence,
                "pcg": st[0].ms_pcg, "g2p": st[0].ms_g2p}
    fused_launches = st[0].kernel_launches + sum(x.kernel_launches for x in st[1:])
    edges = sorted({sc.n[0] for sc in every})
    # the same scenes stepped one at a time through flip_step (the plain per-scene form)
    restart()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for sim in sims:
        sim.step(ksteps)
        sim.sync()
    seq_value = job_rate(npart * ksteps, time.perf_counter() - t0, ws)
    rc = int(max_over_ranks(rc, ws))
    if rank != 0:
        b.close()
        for s_ in sims:
            s_.close()
        return
    peak, peak_kind = read_peaks()
    npart_all = sum(sc.n_particles for sc in every)
    # kernels per step of the timed form.  Fused: the statistics step's count minus its
    # one statistics kernel per scene (7 stage launches, the solves, one G2P since all
    # scenes share a precision).  Per-scene: 7 per scene (2 scans, scatter, P2G,
    # normalisation, divergence, G2P) plus the same solves.
    solves = fused_launches - len(sims) - 7 - 1
    launches_per_step = (fused_launches - len(sims)) if form[0] else 7 * len(sims) + solves
    out = {"metric": "FLIP particle-steps/s", "value": units / (ms / 1e3),
           "unit": "particle-steps/s", "n_gpus": ws, "steps": ksteps, "warmup": args.warmup,
           "ms_per_step": ms / ksteps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": f"batch of {len(every)} dam-break scenes, edges {edges}, "
                                  "fluid fraction 0.2-0.5 by seed", "particles": npart_all,
                      "cells": sum(int(np.prod(sc.n)) for sc in every),
                      "precision": ("mixed: FP32 CG, float-pair solution and residual to 1e-8"
                                    if mixed else "FP32 (float-pair dot products)"),
                      "preconditioner": "multigrid",
                      "form": form_name(*form) + (" (chosen by the autotuner)" if args.autotune
                                                  else ""),
                      "transfer_ctas_per_sm": dict(zip(("p2g", "g2p"), sims[0].transfer_ctas())),
                      "l2": f"inputs larger than L2 ({footprint / 2**30:.2f} GB on the device "
                            "for the batch); no flush",
                      "parallelism": f"scenes sharded over {ws} GPU(s) by the host-side router "
                                     "(longest first to the least-loaded rank), one batch "
                                     "per GPU, no data-path collective"},
           "team_exponent": exponent,
           "cg_iterations_per_scene_step": sum(x.cg_iterations for x in st) / len(st),
           "stages_ms_per_step": stage_ms,
           "stage_roofline": batch_stage_roofline(scenes, nfl, stage_ms, 1, peak),
           "stages_form": "fused (one statistics step)",
           "max_rel_residual": max(x.cg_rel_residual for x in st), "status": rc,
           "gpu_launches": launches_per_step * ksteps, "launches_per_step": launches_per_step,
           "clocks": ck,
           "other_forms": forms,
           "per_scene_sequential": {"value": seq_value, "unit": "particle-steps/s",
                                    "what": "the same scenes, one flip_step call per scene "
                                            "after another (host-timed, synchronised)"}}
    print(json.dumps(out), flush=True)
    b.close()
    for s_ in sims:
        s_.close()


def serve_workload(srv_scenes, max_edge, rate, requests, budget_gb, max_batch, ws=1, rank=0,
                   seed=0, overlap=True, fused=False):
    """Step requests arriving as a Poisson process (mean `rate` per second, uniform
    scene choice) over `srv_scenes` resident dam-break scenes with edges log-uniform
    in [48, max_edge] and fluid fraction 0.2-0.5 (mixed precision), served by the
    continuous-batching server.  Returns this rank's part: latencies, batch sizes,
    particles served, span and set-up figures.  With N ranks the router places each
    scene on one rank."""
    import torch.distributed as dist
    from paper_2404_01931_gb300 import flip as F
    from paper_2404_01931_gb300 import scenes as S
    rng = np.random.default_rng(seed)
    lo, hi = 48, max_edge
    specs = []
    for k in range(srv_scenes):
        n = int(round(np.exp(rng.uniform(np.log(lo), np.log(hi)))))
        specs.append((n, rng.uniform(0.2, 0.5)))
    mine = set(shard_scenes([n ** 3 * f for n, f in specs], ws)[rank])
    t_gen = time.perf_counter()
    srv = F.Server(int(budget_gb * (1 << 30)), max_batch)
    srv.set_overlap(overlap)
    srv.set_fused(fused)
    sid, npart = {}, [0] * len(specs)
    for k, (n, f) in enumerate(specs):
        if k not in mine:
            continue
        side = float(np.sqrt(f))
        sc = S.dam_break(n, side, side, seed=k)
        p = F.default_params(n)
        p.precision = F.FLIP_PREC_MIXED_IR
        p.cg_tol, p.ir_tol = 1e-3, 1e-8
        sid[k] = srv.add_scene(p, *sc.arrays())
        npart[k] = sc.n_particles
    srv.drain()
    t_gen = time.perf_counter() - t_gen
    resident, used = srv.usage()
    # Poisson arrivals, uniform scene choice (the same draws on every rank)
    gaps = rng.exponential(1.0 / rate, requests)
    choice = rng.integers(0, len(specs), requests)
    if ws > 1:
        dist.barrier()
    start = srv.now() + 0.2
    arrivals = start + np.cumsum(gaps)
    reqs = [q for q in range(requests) if int(choice[q]) in mine]
    tickets = [srv.submit(sid[int(choice[q])], float(arrivals[q])) for q in reqs]
    infos = [srv.wait(t) for t in tickets]
    part = dict(lat=[(i.t_done - i.t_arrival) * 1e3 for i in infos],
                batch=[i.batch_size for i in infos],
                failed=int(sum(i.status != F.FLIP_OK for i in infos)),
                served=float(sum(npart[int(choice[q])] for q in reqs)),
                span=(max(i.t_done for i in infos) - float(arrivals[reqs[0]])) if reqs else 0.0,
                resident=resident, used=used, particles=int(sum(npart)), setup=t_gen)
    srv.close()
    return part


def serve_summary(parts, srv_scenes, max_edge, rate, requests, budget_gb, max_batch):
    lat = np.array([v for q in parts for v in q["lat"]])
    span = max(q["span"] for q in parts)
    served = sum(q["served"] for q in parts)
    return {"value": served / span if span > 0 else None, "unit": "particle-steps/s",
            "workload": f"serving: {srv_scenes} resident dam-break scenes, edges log-uniform "
                        f"in [48, {max_edge}], Poisson arrivals at {rate}/s, {requests} "
                        "requests, uniform scene choice, mixed precision",
            "latency_ms": {"p50": float(np.percentile(lat, 50)),
                           "p99": float(np.percentile(lat, 99)), "max": float(lat.max()),
                           "what": "request completion minus arrival (server clock)"},
            "mean_batch": float(np.mean([b for q in parts for b in q["batch"]])),
            "failed": sum(q["failed"] for q in parts),
            "budget_gb": budget_gb, "max_batch": max_batch,
            "resident_scenes": sum(q["resident"] for q in parts),
            "resident_gb": sum(q["used"] for q in parts) / (1 << 30),
            "particles_total": sum(q["particles"] for q in parts),
            "setup_s": round(max(q["setup"] for q in parts), 1), "span_s": span}


def run_serve(args):
    """Step requests arriving as a Poisson process over resident scenes of uneven
    size, served by the continuous-batching server.  With N GPUs the router places
    each scene on one rank (its server), and each rank serves the requests for its
    scenes; latencies and totals are gathered on rank 0."""
    import torch
    import torch.distributed as dist

    import __graft_entry__
    ws, rank, local = dist_setup()
    if rank == 0 or ws == 1:
        __graft_entry__.build()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist.barrier()
        __graft_entry__.build()
    clocks = ClockSampler(local)
    clocks.start()
    part = serve_workload(args.serve, args.serve_max_edge, args.rate, args.requests,
                          args.budget_gb, args.max_batch, ws, rank,
                          overlap=not args.serve_serial, fused=args.serve_fused)
    ck = clocks.stop()
    parts = [part]
    if ws > 1:
        parts = [None] * ws
        dist.all_gather_object(parts, part)
    if rank != 0:
        return
    sv = serve_summary(parts, args.serve, args.serve_max_edge, args.rate, args.requests,
                       args.budget_gb, args.max_batch)
    out = {"metric": "FLIP particle-steps/s", "value": sv["value"], "unit": "particle-steps/s",
           "n_gpus": ws, "steps": args.requests, "warmup": 0,
           "ms_per_step": sv["span_s"] * 1e3 / args.requests, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": sv["workload"], "budget_gb": args.budget_gb,
                      "max_batch": args.max_batch, "resident_scenes": sv["resident_scenes"],
                      "resident_gb": sv["resident_gb"], "particles_total": sv["particles_total"],
                      "setup_s": sv["setup_s"],
                      "l2": f"inputs larger than L2 ({sv['resident_gb']:.1f} GB of resident "
                            "scenes); no flush",
                      "parallelism": f"scenes placed on {ws} GPU(s) by the host-side router "
                                     "(longest first to the least-loaded rank), one server "
                                     "per GPU, no data-path collective"},
           "latency_ms": sv["latency_ms"], "mean_batch": sv["mean_batch"],
           "failed": sv["failed"], "clocks": ck,
           "batches": "one at a time" if args.serve_serial else "overlapped",
           "batch_form": "fused" if args.serve_fused else "per-scene launches"}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--flush-l2", choices=("auto", "always", "never"), default="auto",
                    help="write a buffer twice the L2 before every timed step (auto: when "
                         "the scene's device footprint is under 1 GB)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="pool256", choices=sorted(WORKLOADS))
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-oracle-error", dest="oracle_error", action="store_false",
                    help="skip the per-field comparison of the first step with the oracle")
    ap.add_argument("--batch", type=int, default=0,
                    help="run the batched form: this many dam-break scenes stepped together")
    ap.add_argument("--serve", type=int, default=0,
                    help="run the serving form over this many resident scenes")
    ap.add_argument("--serve-max-edge", type=int, default=192)
    ap.add_argument("--serve-serial", action="store_true",
                    help="serving: one batch at a time instead of overlapped batches")
    ap.add_argument("--serve-fused", action="store_true",
                    help="serving: fused batches instead of per-scene launches inside each")
    ap.add_argument("--rate", type=float, default=2000.0, help="request arrivals per second")
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--budget-gb", type=float, default=180.0)
    ap.add_argument("--max-batch", type=int, default=64)
    ap.add_argument("--no-served", dest="served", action="store_false",
                    help="skip the served sub-measurement of the default line (40 scenes "
                         "<= 96^3 at 2000 requests/s)")
    ap.add_argument("--cfl", type=float, default=0.0,
                    help="adaptive time step with this CFL number (0: fixed dt = 1/240)")
    ap.add_argument("--ppc", type=int, nargs=2, default=(0, 0), metavar=("MIN", "MAX"),
                    help="reseed cells to at least MIN and at most MAX particles (0 0: off)")
    ap.add_argument("--precond", default="mg", choices=["mg", "jacobi", "rbgs"],
                    help="pressure solver: multigrid-preconditioned CG, Jacobi-PCG, or "
                         "red-black Gauss-Seidel iterations (the paper's GPU solver; FP32)")
    ap.add_argument("--mg-smooth", type=int, default=2,
                    help="multigrid red-black sweep pairs before and after the correction")
    ap.add_argument("--batch-fused", action="store_true",
                    help="batch mode without the autotuner: start from the fused form")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="skip the autotuners (one scene: the P2G/G2P launch shapes; "
                         "batch: the solve-team split, the form and the launch shapes)")
    ap.add_argument("--no-surface", dest="surface", action="store_false",
                    help="skip the surface-reconstruction measurement")
    ap.add_argument("--warm-start", action="store_true",
                    help="start every solve from the last solve's pressure (flip_params.warm_start)")
    ap.add_argument("--precision", default=None, choices=["fp32", "mixed"],
                    help="override the workload's precision (fp32: the plain FP32 form)")
    ap.add_argument("--cg-tol", type=float, default=None,
                    help="override the workload's cg_tol (mixed mode: refinement trigger)")
    args = ap.parse_args()
    w = dict(WORKLOADS[args.workload])
    if args.cg_tol is not None:
        w["cg_tol"] = args.cg_tol
    if args.precision is not None:
        w["precision"] = args.precision
    if args.impl == "reference":
        return run_reference(args, w)
    if args.batch:
        return run_batch(args)
    if args.serve:
        return run_serve(args)
    ws, rank, local = dist_setup()
    import torch
    import torch.distributed as dist

    import __graft_entry__
    if rank == 0 or not os.path.exists(os.path.join(ROOT, "paper_2404_01931_gb300", "_lib",
                                                    "libflip_gb300.so")):
        __graft_entry__.build()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist.barrier()
        __graft_entry__.build()
    from paper_2404_01931_gb300 import flip as F

    sc = make_scene(w)
    prm = make_params(w)
    prm.warm_start = 1 if args.warm_start else 0
    prm.cfl = args.cfl
    prm.mg_smooth = args.mg_smooth
    prm.preconditioner = {"mg": F.FLIP_PRECOND_MG, "jacobi": F.FLIP_PRECOND_JACOBI,
                          "rbgs": F.FLIP_PRECOND_RBGS}[args.precond]
    if args.precond != "mg":
        prm.cg_max_iter = 100000
    prm.ppc_min, prm.ppc_max = args.ppc
    sim = F.Simulation(prm, *sc.arrays())
    stream = torch.cuda.ExternalStream(sim.stream)
    np_ = sc.n_particles
    # the first step of the seeded scene, kept for the comparison with the oracle
    # (computed after the timed region); it counts as a warm-up step
    first = None
    want_err = (args.oracle_error and rank == 0 and ws == 1 and not (args.ppc[0] or args.ppc[1])
                and args.cfl == 0 and not args.warm_start and args.precond == "mg")
    warm_left = args.warmup
    if want_err and warm_left > 0:
        sim.step(1, stats=True)
        first = first_step_fields(sim, F)
        warm_left -= 1
    # the launch shapes of P2G and G2P, chosen on this scene by the autotuner (6
    # untimed steps); the scene then starts again from its seeded particles and
    # takes the warm-up steps, so the timed steps are those of the run without it
    shapes = None
    if args.autotune and not (args.ppc[0] or args.ppc[1]) and args.cfl == 0:
        shapes = sim.autotune_transfers(1)
        ids = sim.read(F.PID)
        F.flip_write_particles(sim.h, *[np.ascontiguousarray(a[ids]) for a in sc.arrays()])
        warm_left = args.warmup
    if warm_left > 1:
        sim.step(warm_left - 1)
    if warm_left > 0:
        sim.step(1, stats=True)  # also sizes the library's pool of timing events
    sim.sync()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    # scenes whose device footprint is under 1 GB could be served from the 126 MB L2
    # across steps: then a buffer twice the L2 is written before every timed step
    # (outside the step's own CUDA events, which time it)
    footprint = F.flip_footprint_bytes(prm, np_)
    flush = args.flush_l2 == "always" or (args.flush_l2 == "auto" and footprint < (1 << 30))
    if flush:
        scrub = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device="cuda")
        st = F.FlipStats()
        step_ms = []
        last = [f for f, _ in F.FlipStats._fields_ if not (f.startswith("ms_") or f in (
            "cg_iterations", "ir_iterations", "kernel_launches", "particles_added",
            "particles_removed", "steps"))]
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                scrub.zero_()
            rc, s1 = sim.step(1, stats=True)
            step_ms.extend(sim.step_times().tolist())
            for f, _ in F.FlipStats._fields_:
                setattr(st, f, getattr(s1, f) if f in last else getattr(st, f) + getattr(s1, f))
        torch.cuda.synchronize()
        step_ms = np.asarray(step_ms, np.float64)
        ms_local = float(step_ms.sum())
    else:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc, st = sim.step(args.steps, stats=True)
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms = sim.step_times()
        ms_local = e0.elapsed_time(e1)
    if ws > 1:
        dist.barrier()
    ck = clocks.stop()
    ms = max_over_ranks(ms_local, ws)
    np_ = st.n_particles if args.ppc[0] or args.ppc[1] else np_
    value = job_rate(np_ * args.steps, ms_local / 1e3, ws)

    # end to end: host (pinned) buffers in, one step, host buffers out, every step
    e2e = None
    if args.e2e_steps > 0 and not (args.ppc[0] or args.ppc[1]):
        host = [torch.empty(np_, dtype=torch.float32, pin_memory=True) for _ in range(6)]
        F.flip_read_particles(sim.h, *host)
        sim.sync()
        if ws > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            F.flip_write_particles(sim.h, *host)
            sim.step(1)
            F.flip_read_particles(sim.h, *host)
        el = time.perf_counter() - t0
        e2e = {"value": job_rate(np_ * args.e2e_steps, el, ws), "unit": "particle-steps/s",
               "h2d_bytes_per_step": 24 * np_, "d2h_bytes_per_step": 24 * np_,
               "steps": args.e2e_steps}

    # energy diagnostic (Sec. 4, Fig. 10), outside the timed region: 24 B per
    # particle; each call ends with a host synchronisation, included in its time
    diag = None
    if rank == 0:
        m = prm.rho * prm.dx ** 3 / 8
        sim.energy(m)
        t = []
        for _ in range(5):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            energy = sim.energy(m)
            b.record(stream)
            b.synchronize()
            t.append(a.elapsed_time(b))
        diag = {"energy_ms": min(t), "energy_bytes": 24 * np_, "energy_total": energy[2]}

    # surface reconstruction (Sec. 3.3) of the final state on the simulation grid,
    # outside the timed region: scalar field (CUDA events on the shared stream) and
    # marching cubes + normals (ends with a host synchronisation, included)
    surf = None
    if rank == 0 and args.surface:
        sp = F.surface_default_params(prm)
        sfc = F.Surface(sp, stream=sim.stream)
        best = None
        for _ in range(3):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record(stream)
            sfc.sdf(sim)
            ev[1].record(stream)
            nv, nt = sfc.mesh()
            ev[2].record(stream)
            ev[2].synchronize()
            t = (ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]))
            best = t if best is None or sum(t) < sum(best) else best
        corners = (w["n"] + 1) ** 3
        surf = {"sampling_corners": corners, "radius_dx": 0.5, "search_radius_dx": 2.0,
                "sdf_ms": best[0], "mesh_ms": best[1], "n_vertices": nv, "n_triangles": nt,
                "corners_per_s": corners / ((best[0] + best[1]) / 1e3)}
        sfc.close()

    if rank == 0:
        peak, peak_kind = read_peaks()
        nfl = st.n_fluid_cells
        if diag:
            diag["energy_frac_of_measured_hbm"] = diag["energy_bytes"] / (diag["energy_ms"] / 1e3) / 1e9 / peak
        mixed = w["precision"] == "mixed"
        # the method's algorithmic bytes of the solves (47 B per fluid cell per CG
        # iteration + 40 B per refinement) and the build's model that also counts
        # the V-cycle's passes
        method_bytes = nfl * (METHOD_PCG_BYTES_PER_ITER * st.cg_iterations
                              + (METHOD_IR_BYTES_PER_OUTER * st.ir_iterations if mixed else 0))
        pcg_bytes = nfl * (MG_PCG_BYTES_PER_ITER * st.cg_iterations
                           + (MG_IR_BYTES_PER_OUTER * st.ir_iterations
                              + MG_IR_BYTES_PER_SOLVE * args.steps if mixed else 0))
        stage_ms = {"bin": st.ms_bin, "p2g": st.ms_p2g, "divergence": st.ms_divergence,
                    "pcg": st.ms_pcg, "g2p": st.ms_g2p}
        t_pcg = st.ms_pcg / 1e3
        achieved = method_bytes / t_pcg / 1e9 if t_pcg > 0 else None
        achieved_vc = pcg_bytes / t_pcg / 1e9 if t_pcg > 0 else None
        traffic, traffic_note = (recorded_pcg_traffic() if args.workload == "pool256"
                                 else (None, "captured for the 256^3 pool only"))
        out = {
            "metric": "FLIP particle-steps/s", "value": value, "unit": "particle-steps/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w["desc"], "grid": [w["n"]] * 3, "particles": np_,
                       "precision": "mixed: FP32 PCG with float-pair (~48-bit) solution and "
                       "residual replacement, FP64 right-hand side and result" if mixed
                       else "FP32 (float-pair dot products)",
                       "ir_tol": w["ir_tol"], "cg_tol": w["cg_tol"], "dt": 1 / 240,
                       "flip_ratio": 0.95, "seed": 0,
                       "parallelism": f"{ws} independent replica(s), one per GPU",
                       "l2": (f"L2 flushed before every timed step (a {2 * L2_BYTES >> 20} MB "
                              f"buffer written; device footprint {footprint / 2**20:.0f} MB); "
                              "value from the steps' own CUDA events") if flush else
                             (f"inputs larger than L2 (device footprint {footprint / 2**30:.2f} GB); "
                              "no flush"),
                       "pressure_start": "last solve's pressure (warm start)" if args.warm_start
                       else "zero (cold start)",
                       "mg_smooth": args.mg_smooth, "solver": args.precond,
                       "transfer_ctas_per_sm": dict(zip(("p2g", "g2p"), sim.transfer_ctas()),
                                                    chosen_by="autotuner (6 untimed steps)"
                                                    if shapes else "defaults"),
                       "time_step": f"adaptive, CFL number {args.cfl}" if args.cfl > 0
                       else "fixed 1/240",
                       "reseeding": f"{args.ppc[0]}..{args.ppc[1]} particles per cell"
                       if args.ppc[0] or args.ppc[1] else "off"},
            "dt_last": st.dt_last, "particles_added": st.particles_added,
            "particles_removed": st.particles_removed,
            "stages_ms_per_step": {k: v / args.steps for k, v in stage_ms.items()},
            "cg_iterations_per_step": st.cg_iterations / args.steps,
            "ir_iterations_per_step": st.ir_iterations / args.steps,
            "rel_residual": st.cg_rel_residual, "rel_divergence": st.rel_divergence,
            "n_fluid_cells": nfl, "status": rc,
            "latency_ms": {"p50": float(np.percentile(step_ms, 50)) if len(step_ms) else None,
                           "p99": float(np.percentile(step_ms, 99)) if len(step_ms) else None,
                           "max": float(step_ms.max()) if len(step_ms) else None,
                           "mean": float(step_ms.mean()) if len(step_ms) else None,
                           "samples": int(len(step_ms)),
                           "what": "device time of each timed step (CUDA events around the "
                                   "step's kernels on the simulation's stream)"},
            "roofline": {"kernel": "k_pcg_mg (persistent multigrid-preconditioned CG, "
                                   "whole solve per launch)",
                         "bound": "hbm", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": (achieved / peak) if achieved else None,
                         "frac_survey": (achieved / peak) if achieved else None,
                         "byte_model": f"{METHOD_PCG_BYTES_PER_ITER} B per fluid cell per CG "
                                       f"iteration + {METHOD_IR_BYTES_PER_OUTER} B per fluid "
                                       "cell per outer refinement",
                         "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                         "nominal_peak": NOMINAL_HBM_GBS,
                         "frac_of_nominal": (achieved / NOMINAL_HBM_GBS) if achieved else None,
                         "algorithmic_bytes_per_launch": method_bytes / args.steps,
                         "with_vcycle_bytes": {
                             "bytes_per_launch": pcg_bytes / args.steps,
                             "achieved": achieved_vc,
                             "frac": (achieved_vc / peak) if achieved_vc else None,
                             "model": f"{MG_PCG_BYTES_PER_ITER} B per fluid cell per iteration "
                                      "including the V-cycle's passes"},
                         "traffic": traffic, "traffic_source": traffic_note,
                         "solver_source_hash": solver_source_hash()},
            "stage_roofline": stage_roofline(w, np_, nfl, stage_ms, args.steps, peak),
            "gpu_launches": st.kernel_launches,
            "diagnostics": diag,
            "surface": surf,
            "clocks": ck,
            "e2e": e2e,
        }
        if not args.no_cpu_baseline and ws == 1:
            out["cpu_baseline"] = cpu_baseline(w)
        if first is not None:
            out["error_vs_oracle"] = error_vs_oracle(w, sc, first)
    if rank == 0 and ws == 1 and args.served:
        # the served form beside the headline (same run, after the single scene is freed)
        sim.close()
        part = serve_workload(40, 96, 2000.0, 2000, 180.0, 64)
        out["served"] = serve_summary([part], 40, 96, 2000.0, 2000, 180.0, 64)
        part = serve_workload(40, 96, 2000.0, 2000, 180.0, 64, overlap=False)
        one = serve_summary([part], 40, 96, 2000.0, 2000, 180.0, 64)
        out["served"]["one_batch_at_a_time"] = {k: one[k] for k in ("value", "latency_ms",
                                                                  "mean_batch", "failed")}
    if rank == 0:
        print(json.dumps(out), flush=True)
    sim.close()
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
