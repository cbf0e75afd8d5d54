"""Host logic of bench.py, on CPU.

* The reference arm (the FP64 oracle timed on the host cores) prints one JSON
  line with the contract's keys on rank 0, and nothing on the other ranks.
* With N replicas the job's time is the slowest rank's: max_over_ranks under a
  two-rank gloo process group, and the whole-job rate from it.
* The clock record: median SM clock, maximum clock and every throttle reason seen
  in nvidia-smi's samples; "unsampled" where nvidia-smi is missing.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(args, env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                          env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_line():
    r = run_bench(["--impl", "reference", "--workload", "emc32", "--n-data", "200", "--steps",
                   "2", "--warmup", "1"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "pairs/s" and d["higher_is_better"]
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1
    assert d["config"]["workload"].startswith("emc32")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert "rotations" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "pairs/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_do_nothing():
    r = run_bench(["--impl", "reference", "--workload", "emc32", "--n-data", "200", "--steps",
                   "1", "--warmup", "0"], {"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 2.0 + 3.0 * rank  # the ranks' own times: 2 ms and 5 ms
    job_ms = bench.max_over_ranks(dist, ms, "cpu")
    rate = bench.whole_job_rate(world, 1000, job_ms)
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"ms": job_ms, "rate": rate}, f)


def test_max_over_ranks_gloo(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    for rank in range(world):
        d = json.loads((tmp_path / f"r{rank}.json").read_text())
        assert d["ms"] == 5.0
        assert d["rate"] == pytest.approx(2 * 1000 / 5e-3)


def test_no_process_group_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(None, 3.25, "cpu") == 3.25
    assert bench.whole_job_rate(1, 500, 2.0) == pytest.approx(250000.0)


def test_clock_summary_parses_samples():
    sys.path.insert(0, ROOT)
    import bench
    c = bench.ClockSampler(0)
    # index, sm, max sm, power, active mask, hw, hw thermal, sw thermal, sw power cap
    c.rows = [["0", "2070", "2070", "900.1", "0x0", "Not Active", "Not Active", "Not Active",
               "Not Active"],
              ["0", "1980", "2070", "1390.5", "0x4", "Not Active", "Not Active", "Not Active",
               "Active"],
              ["0", "2070", "2070", "1201.0", "0x0", "Not Active", "Not Active", "Not Active",
               "Not Active"],
              ["garbled line"]]
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 4
    c.rows[0][6] = "Active"  # a thermal slowdown anywhere in the region is reported
    assert bench.ClockSampler.summary(c)["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_clock_sampler_without_nvidia_smi(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("PATH", "/nonexistent")
    with bench.ClockSampler(0) as c:
        pass
    assert c.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
