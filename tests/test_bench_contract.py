"""bench.py's reference arm (the FP64 CPU oracle timed on the host cores) on a
tiny particle sample: one JSON line with the benchmark's keys, and, under a
multi-rank launch, output from rank 0 only (the other ranks exit 0 silently).
Runs without a GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(*args, env=None):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args],
                          capture_output=True, text=True, timeout=300, cwd=ROOT,
                          env=dict(os.environ, **(env or {})))


def test_reference_arm_prints_one_contract_line():
    r = _bench("--impl", "reference", "--steps", "2", "--warmup", "1", "--cpu-particles", "2")
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["higher_is_better"] is True and d["scaling"] == "weak"
    assert d["vs_baseline"] is None and d["data"] == "synthetic" and d["dtype"] == "f64"
    assert "workload" in d["config"] and d["config"]["particles"] == 1048576
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert cb["unit"] == d["unit"] and "2 of 1048576" in cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    r = _bench("--impl", "reference", "--steps", "1", "--warmup", "1", "--cpu-particles", "2",
               env={"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_traffic_hash_ignores_comments_but_not_code():
    sys.path.insert(0, ROOT)
    import bench
    src = 'int a = b / c; // note\n/* block\n comment */ const char* s = "// kept /* kept */";\n'
    assert bench.code_only(src) == 'int a = b / c; const char* s = "// kept /* kept */";'
    assert bench.code_only("x = 1; // one") == bench.code_only("x  =  1;\n/* other */")
    assert bench.code_only("x = 1;") != bench.code_only("x = 2;")
    assert bench.code_only("c = '/'; d = '*';") == "c = '/'; d = '*';"
