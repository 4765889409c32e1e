"""bench.py's reference arm (the CPU oracle on the benchmark's metric) runs
without a GPU: one JSON line with the contract's keys on rank 0, nothing
and exit 0 on the other ranks."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(args, env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, capture_output=True, text=True,
                          env=env, timeout=600, cwd=ROOT)


def test_reference_arm_prints_one_line():
    r = run(["--impl", "reference", "--steps", "2", "--warmup", "3", "--workload", "gauss_poly1_1e4"])
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "events/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["config"]["workload"] == "gauss_poly1_1e4"


def test_reference_arm_other_ranks_exit_quietly():
    r = run(["--impl", "reference", "--steps", "1"], {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_clock_summary_parses_samples_and_reasons():
    sys.path.insert(0, ROOT)
    import bench

    c = bench.ClockSampler(0)
    c.out = "\n".join([
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1350.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 1980, 2070, 1400.0, 0x4, Active, Not Active, Not Active, Active",
        "0, [N/A], 2070, [N/A], 0x0, Not Active, Not Active, Not Active, Not Active",
    ])
    s = c.summary()
    assert s["sm_mhz"] == 2055.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 4
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"]
    c.out = None
    assert c.summary()["reasons"] == ["nvidia-smi unavailable"]
