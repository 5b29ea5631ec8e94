"""The reference arm of bench.py (the oracle timed on the host cores, on a
bounded sample of the 2e7-track shower) prints the one JSON line the bench
contract names, and ranks other than 0 exit without work."""
import json
import os
import subprocess
import sys

REPO = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ARGS = ["--impl", "reference", "--steps", "1", "--warmup", "1", "--cpu-sample-tracks", "2000"]


def run(env=None):
    return subprocess.run([sys.executable, "bench.py", *ARGS], cwd=REPO, capture_output=True, text=True,
                          timeout=600, env=env)


def test_reference_arm_prints_the_contract_line():
    p = run()
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["unit"] == "pairs/s" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["steps"] == 1 and line["warmup"] == 1
    assert line["config"]["pairs_per_step"] == 2 * 2000 * 160
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": "pairs/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_without_work():
    p = run(dict(os.environ, RANK="1"))
    assert p.returncode == 0 and p.stdout.strip() == ""
