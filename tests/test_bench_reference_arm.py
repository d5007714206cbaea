"""The reference arm of bench.py on the CPU: `--impl reference` times the
oracle (the only reference this method has) and prints one JSON line on rank
0 with the same metric, unit and workload as the GPU arm, a cpu_baseline
describing the run, and an e2e with no host/device traffic; other ranks exit
without output."""
import json
import os
import subprocess
import sys
from pathlib import Path

ROOT = Path(__file__).resolve().parent.parent
N = 40_000  # the configuration's stream scaled down (the arm itself runs at n = 2,000,000)


def run(extra_env=None):
    env = dict(os.environ, **(extra_env or {}))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "3",
                        "--n", str(N)],
                       cwd=str(ROOT), env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return [json.loads(line) for line in r.stdout.splitlines() if line.startswith("{")]


def test_reference_arm_line():
    import bench

    lines = run()
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == "ms" and d["higher_is_better"] is False
    assert d["value"] > 0 and d["ms_per_step"] == d["value"] and d["steps"] == 2 and d["warmup"] == 3
    assert d["config"] == bench.config_of(N)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_other_ranks_print_nothing():
    assert run({"RANK": "1", "WORLD_SIZE": "2"}) == []


def test_timed_schedule_stays_on_the_configuration():
    import bench

    # W = 3, K = 8: the configuration's steps t = 5..12 once
    assert bench.timed_schedule(3, 8) == [list(range(4, 12))]
    # W = 5, K = 20: t = 7..12 replayed from the post-warm-up checkpoint
    segs = bench.timed_schedule(5, 20)
    assert [len(s) for s in segs] == [6, 6, 6, 2]
    assert all(s[0] == 6 for s in segs) and max(max(s) for s in segs) == bench.LFR_STEPS - 1
    assert sum(len(s) for s in segs) == 20
