"""The reference arm of bench.py on the host: `--impl reference` times the FP64
oracle on the headline workload (two 2048^2 resonators, a few bounces each
per step, the oracle's per-call set-up timed apart) and prints one JSON line
with the same metric, unit and workload configuration as the GPU arm, the
oracle described as the CPU baseline, and an end-to-end figure with no
host-device traffic."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    sys.path.insert(0, ROOT)
    import bench

    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["higher_is_better"] is True and line["n_gpus"] == 1
    assert line["steps"] == 1 and line["warmup"] == 0 and line["value"] > 0.0
    assert line["config"] == bench.config_block()
    assert line["bounces_per_step"] == bench.REF_BOUNCES_PER_STEP and line["oracle_setup_s_per_call"] > 0.0
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1 and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
