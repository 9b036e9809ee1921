"""The bench's JSON contract on the reference arm, which runs on the host
cores alone (the FP64 oracle, timed on whole measured steps): one line with
the metric, the whole-job value, the configuration the GPU arm prints too,
and the cpu_baseline and e2e objects; the steps it claims fit inside the
run's own wall clock. No GPU needed."""
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    t0 = time.perf_counter()
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "2", "--warmup", "1"], capture_output=True, text=True,
                         cwd=ROOT, timeout=600)
    wall = time.perf_counter() - t0
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "force interactions/s" and d["unit"] == "interactions/s"
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 1
    # measured, not extrapolated: the claimed steps fit in the run
    assert d["ms_per_step"] * 1e-3 * d["steps"] < wall
    assert d["higher_is_better"] is True and d["scaling"] in ("weak", "strong")
    assert d["vs_baseline"] is None and d["dtype"] == "f64"
    assert d["config"]["workload"].startswith("plummer_1m")
    sys.path.insert(0, ROOT)
    import bench

    wl = bench.workload("plummer_1m")
    assert d["config"] == bench.bench_config(wl, 1)  # the GPU arm's config object
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert cb["cpu_model"] and cb["nproc"] >= 1 and cb["group_stride"] == 1
    assert cb["unit"] == d["unit"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
