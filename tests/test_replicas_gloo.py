"""Multi-GPU is replicas only: each rank runs an independent copy of the
workload with its own Philox seed and no data-path collective; the job
value is all ranks' particle-steps over the slowest rank's time. The
rank-level logic is exercised here with world_size 2 on gloo (CPU)."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import sys

    import torch.distributed as td

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    td.init_process_group("gloo", rank=rank, world_size=world)
    p = bench.replica_params(bench.workload("smallest"), rank)
    local_ms = 100.0 + 50.0 * rank
    mx = bench.max_over_ranks(local_ms)
    val = bench.aggregate_value(p["n_particles"], 5, world, mx)
    q.put((rank, p["seed"], mx, val))
    td.destroy_process_group()


def test_two_replicas_on_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    seeds = [r[1] for r in res]
    assert seeds == [0, 1]
    assert all(r[2] == 150.0 for r in res)          # max over ranks
    assert all(abs(r[3] - 2 * 4096 * 5 / 0.150) < 1e-6 for r in res)


def test_single_rank_helpers_without_process_group():
    import bench

    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.replica_params({"seed": 7}, 3)["seed"] == 10


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference times the oracle on the host cores and prints
    one JSON line with the contract's keys (a small sample here)."""
    import json
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--cpu-mesh", "8"], capture_output=True, text=True, timeout=300,
                         cwd=root, check=True).stdout
    lines = [l for l in out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert "workload" in d["config"]


def test_clock_summary_reports_median_max_and_active_reasons():
    """The clock record beside each bench number: median SM clock under load,
    the maximum clock, and every throttle reason seen active (nvidia-smi CSV
    rows, synthetic here)."""
    import bench

    s = bench.ClockSampler(0)
    assert s.summary()["samples"] == 0 and s.summary()["reasons"] == ["clock samples unavailable"]
    na, a = "Not Active", "Active"
    s.rows = [["0", "2070", "2070", "900.5", "0x0", na, na, na, na],
              ["0", "1980", "2070", "1400.0", "0x4", na, na, na, a],
              ["0", "2070", "2070", "1395.1", "0x0", na, na, na, na]]
    d = s.summary()
    assert d["sm_mhz"] == 2070.0 and d["sm_max_mhz"] == 2070.0 and d["samples"] == 3
    assert d["reasons"] == ["sw_power_cap"]
    s.rows.append(["0", "1500", "2070", "1200.0", "0x48", a, na, a, na])
    assert bench.ClockSampler.summary(s)["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]
