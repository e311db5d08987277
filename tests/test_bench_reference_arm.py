"""`bench.py --impl reference` on CPU: one JSON line with the contract's keys,
the oracle timed on the host cores, no GPU touched."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1
    assert d["higher_is_better"] is True and d["value"] > 0
    assert d["unit"] == "guided samples/s" and d["config"]["rays"] == 1_602_720
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # value and ms_per_step are measured: the guided samples the step made over its wall time
    rate = d["guided_samples_per_step"] / (d["ms_per_step"] / 1e3)
    assert abs(d["value"] - rate) <= 1e-9 * rate
    assert d["frame_rate_projected"]["value"] > 0 and d["frame_rate_projected"]["how"]
    # the same config dict as the GPU arm prints
    for k in ("workload", "rays", "records", "bins", "grid", "svo_depth", "svo_nodes", "l2", "parallelism", "streams"):
        assert k in d["config"], k
    assert d["config"]["records"] == 1_646_633 and d["config"]["svo_nodes"] > 0
