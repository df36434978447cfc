"""bench.py keeps its JSON-line contract: one line with the metric, the
device-timed value, the roofline, the end-to-end figure, the clocks, the
launch count and the CPU baseline (a small workload, run as a subprocess)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _run(*args):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1, r.stdout
    return json.loads(lines[0])


def test_single_graph_line():
    d = _run("--workload", "er10k", "--steps", "3", "--warmup", "3", "--e2e-steps", "1",
             "--cpu-seconds", "0.2", "--multi", "2")
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "roofline", "clocks", "e2e", "gpu_launches", "cpu_baseline"):
        assert k in d, k
    assert d["value"] > 0 and d["n_gpus"] == 1 and d["steps"] == 3 and d["warmup"] >= 3
    assert d["config"]["workload"] == "er10k"
    r = d["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in r, k
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and 0 < r["frac"]
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-9
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    c = d["cpu_baseline"]
    assert c["kind"] == "oracle" and c["cores"] >= 1 and c["value"] > 0
    assert c["gpu_result_equals_oracle"] is True
    par = d["cpu_parallel"]
    assert par["value"] > 0 and par["cores"] >= 1 and par["result_equals_oracle"] is True
    assert d["gpu_launches"] == 3
    assert d["config"]["multi_seed"]["k"] == 2
    # the timed solve starts from the CSR; B0 over its time cannot pass the peak
    assert r["alg_bytes_per_launch"] == 4 * d["config"]["arcs"] + 4 * (d["config"]["n"] + 1)
    assert r["frac"] <= 1.0
    assert r["work_bytes"] >= r["alg_bytes_per_launch"]
    cr = d["config"]["create"]
    for k in ("default", "full_rows", "round0_structures"):
        assert cr[k]["create_s"] > 0 and cr[k]["create_plus_first_solve_ms"] > 0
    am = d["config"]["amortized"]
    assert am["same_result"] is True and am["per_solve_ms_p50"] > 0


def test_single_graph_line_with_legs():
    d = _run("--workload", "er10k", "--steps", "3", "--warmup", "3", "--e2e-steps", "0",
             "--no-cpu-baseline", "--multi", "0", "--legs", "batch,serve,tc", "--batch-count", "64",
             "--pool", "8", "--requests", "400", "--serve-check", "32")
    b = d["batch4096"]
    assert b["graphs"] == 64 and b["graphs_per_s"] > 0
    assert b["standalone_check"]["all_equal"] is True
    s = d["serve"]
    assert s["pool"] == 8 and s["requests"] == 400
    assert s["served_graphs_per_s"] > 0 and s["sequential_graphs_per_s"] > 0
    for k in ("saturated", "poisson_0.5", "poisson_0.8", "poisson_1.0"):
        assert s[k]["p99_ms"] >= s[k]["p50_ms"] > 0
    assert s["standalone_check"]["all_equal"] is True
    t = d["tiles_tc"]
    assert t["multi_seed_tc"]["results_equal_csr"] is True
    assert set(t["multi8_ms"]) == {"csr", "rows_tc_b1", "tc_bits_fp16", "tc_b1", "tc_int8",
                                   "tc_fp16"}
    assert t["autotune_multi_form"] in ("csr", "rows_tc_b1")
