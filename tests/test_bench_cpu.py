"""bench.py on CPU: the reference arm's JSON line (the oracle, small sizes) and
the host-side helpers of the GPU arm."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "3000", "--m", "1500",
           "--steps", "2", "--warmup", "3"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT,
                       env={**os.environ, "CUDA_VISIBLE_DEVICES": ""})
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["steps"] == 2 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["unit"] == "queries/s" and d["higher_is_better"] is True and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["n_users"] == 3000 and d["config"]["n_items"] == 1500 and "workload" in d["config"]


def test_result_sizes_buckets():
    sys.path.insert(0, ROOT)
    import bench
    offs = np.array([0, 0, 5, 5, 45, 10045, 20046], dtype=np.int64)   # sizes 0, 5, 0, 40, 10000, 10001
    out = bench.result_sizes(offs)
    assert out["queries"] == 6 and out["total"] == 20046 and out["max"] == 10001
    assert out["n_0-0"] == 2 and out["ids_0-0"] == 0
    assert out["n_1-32"] == 1 and out["ids_1-32"] == 5
    assert out["n_33-8192"] == 1 and out["ids_33-8192"] == 40
    assert out["n_8193+"] == 2 and out["ids_8193+"] == 20001
    assert bench.result_sizes(None) is None
