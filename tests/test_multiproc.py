"""The multi-process path of bench.py (one replica per GPU, no collective on the
data path): rank setup from the environment, the slowest rank's time and the
whole-job rate over two gloo ranks on the CPU."""
import os
import socket
import subprocess
import sys
import textwrap

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import os, sys, json
    sys.path.insert(0, {root!r})
    import torch.distributed as dist
    import bench
    ws, rank, local = bench.dist_setup()
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    t = 1.0 + rank                      # rank 1 is the slower one
    units = 100 * (rank + 1)
    out = dict(ws=ws, rank=rank, local=local, tmax=bench.max_over_ranks(t, ws),
               total=bench.sum_over_ranks(units, ws), rate=bench.job_rate(units, t, ws))
    dist.barrier()
    dist.destroy_process_group()
    print(json.dumps(out))
""")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_two_gloo_ranks_reduce_time_and_rate():
    import json
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", CHILD.format(root=ROOT)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    for r, o in enumerate(outs):
        assert (o["ws"], o["rank"], o["local"]) == (2, r, r)
        assert o["tmax"] == 2.0                     # the slowest rank's time
        assert o["total"] == 300.0                  # units summed over the ranks
        assert o["rate"] == 150.0                   # whole-job units per second


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_rate(100, 2.0, 1) == 50.0


def test_router_partitions_and_balances():
    """The host-side router of batched and served scenes: every scene on exactly one
    rank, the plan deterministic, and each rank's load within the largest scene of
    the mean (longest-first greedy)."""
    sys.path.insert(0, ROOT)
    import bench
    import numpy as np
    rng = np.random.default_rng(5)
    w = [int(v) for v in rng.integers(1, 1000, size=64)]
    for n in (1, 2, 3, 4, 8):
        plan = bench.shard_scenes(w, n)
        assert plan == bench.shard_scenes(w, n)
        flat = sorted(i for p in plan for i in p)
        assert flat == list(range(len(w)))
        loads = [sum(w[i] for i in p) for p in plan]
        assert max(loads) - sum(w) / n <= max(w)
    assert bench.shard_scenes([5, 5], 4) == [[0], [1], [], []]
    assert bench.shard_scenes([], 2) == [[], []]


ROUTER_CHILD = textwrap.dedent("""
    import os, sys, json
    sys.path.insert(0, {root!r})
    import torch.distributed as dist
    import bench
    from paper_2404_01931_gb300 import scenes as S
    ws, rank, local = bench.dist_setup()
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    every = S.batch_scenes(12, seed=0)
    mine = bench.shard_scenes([sc.n_particles for sc in every], ws)[rank]
    parts = [None] * ws
    dist.all_gather_object(parts, mine)
    units = sum(every[i].n_particles for i in mine)
    out = dict(rank=rank, mine=mine, parts=parts, total=bench.sum_over_ranks(units, ws),
               want=sum(sc.n_particles for sc in every))
    dist.barrier()
    dist.destroy_process_group()
    print(json.dumps(out))
""")


def test_two_gloo_ranks_shard_the_batch():
    """Each rank takes its share of the batch from the same plan, computed locally."""
    import json
    port = _free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", ROUTER_CHILD.format(root=ROOT)],
                                      env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                      text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=180)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    a, b = outs
    assert a["parts"] == b["parts"] == [a["mine"], b["mine"]]
    assert sorted(a["mine"] + b["mine"]) == list(range(12)) and not set(a["mine"]) & set(b["mine"])
    assert a["total"] == b["total"] == a["want"]          # every particle counted once


def test_clock_summary_from_nvidia_smi_lines():
    """The bench's clock record: median SM clock, maximum clock, and the throttle
    reasons seen active (a run with hw or thermal slowdown is rejected; sw_power_cap is
    kept and noted)."""
    sys.path.insert(0, ROOT)
    import bench
    na = "Not Active"
    lines = [f"0, 2070, 2070, 950.1, 0x0000000000000000, {na}, {na}, {na}, {na}",
             f"0, 1980, 2070, 1390.0, 0x0000000000000004, {na}, {na}, {na}, Active",
             f"0, 2070, 2070, 1001.2, 0x0000000000000000, {na}, {na}, {na}, {na}",
             "garbage", "0, [N/A], 2070, 0, 0x0, x, x, x, x"]
    s = bench.ClockSampler.summarize(lines)
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                 "samples": 3}
    s = bench.ClockSampler.summarize([f"0, 1500, 2070, 800, 0x8, Active, {na}, Active, {na}"])
    assert s["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"] and s["sm_mhz"] == 1500.0
    assert bench.ClockSampler.summarize([])["sm_mhz"] is None


def test_reference_arm_json_line():
    """`bench.py --impl reference` (the FP64 oracle on the host cores) prints one JSON
    line with the contract's keys; it needs no GPU."""
    import json
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "dam32", "--steps", "2", "--warmup", "1"], cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    d = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert (d["steps"], d["warmup"], d["n_gpus"]) == (2, 1, 1)
