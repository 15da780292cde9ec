"""The JSON line of bench.py's reference arm (the CPU oracle; runs without a GPU): every key
of the bench contract is present with the right kind of value."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _line(*extra):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--cpu-sample-atoms", "24", *extra],
                         capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert out.returncode == 0, out.stderr
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


def test_reference_line_has_the_contract_keys():
    for method in ("rsscs", "nl"):
        d = _line("--method", method)
        for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                  "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
            assert k in d, k
        assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
        assert d["unit"] == "solves/s" and d["steps"] == 1 and d["warmup"] == 0
        assert d["config"]["workload"] == "finite8000"
        # the reference arm describes the workload exactly as the GPU arm does
        assert d["config"] == bench.workload_config("finite8000", method, 8000, 1)
        assert d["config"]["method"] == ("MBD-NL" if method == "nl" else "MBD@rsSCS")
        cb = d["cpu_baseline"]
        assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
        e2e = d["e2e"]
        assert e2e["value"] == d["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
