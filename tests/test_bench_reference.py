"""The reference arm of bench.py (the oracle on the host cores) on a small
sample: one JSON line with the keys and types of the benchmark contract,
the GPU line's workload config, and a value that is the dofs solved per
second of solve time."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1", "--oracle-cells", "3"], cwd=ROOT, capture_output=True, text=True,
                       timeout=600, env=dict(os.environ, CUDA_VISIBLE_DEVICES=""))
    assert r.returncode == 0, r.stderr[-500:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    for key, typ in (("metric", str), ("value", float), ("unit", str), ("ms_per_step", float),
                     ("higher_is_better", bool), ("scaling", str), ("dtype", str), ("data", str),
                     ("config", dict), ("cpu_baseline", dict), ("e2e", dict)):
        assert isinstance(d[key], typ), key
    assert d["vs_baseline"] is None and d["value"] > 0
    assert d["config"]["ndof"] == 32 ** 3 * 125 and d["config"]["mesh"] == [32, 32, 32]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and "3^3" in cb["sample"]
    assert cb["apply_gdofs"] > 0 and cb["lu_sweep_gdofs"] > 0     # the oracle's SpMV and dense-LU sweep
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # value = dofs solved / solve time
    assert abs(3 ** 3 * 125 / (d["ms_per_step"] / 1e3) / 1e9 - d["value"]) <= 0.01 * d["value"]
