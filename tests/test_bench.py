"""The benchmark's own contract, checked on the CPU: the reference arm's JSON
line, the clock record's throttle reasons, and the binding's refusal to run
without the CUDA library (there is no CPU fallback)."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_binding_refuses_to_run_without_the_library():
    code = ("import paper_2507_10070_b300._abi as a; a.LIB_PATH = '/nonexistent/libann.so'\n"
            "import paper_2507_10070_b300 as ann, numpy as np\n"
            "try:\n"
            "    ann.knn_exact(np.zeros((4, 4), np.uint8), np.zeros((1, 4), np.uint8), 1)\n"
            "except ImportError as e:\n"
            "    print('refused:', 'no CPU fallback' in str(e))\n")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True,
                         timeout=120)
    assert out.stdout.strip() == "refused: True", out.stderr


def test_clock_record_flags_throttle_reasons():
    clk = bench.ClockSampler(0)
    clk.lines = ["2032, 2032, 700.1, Not Active, Not Active, Not Active, Not Active",
                 "2032, 2032, 900.5, Not Active, Not Active, Not Active, Active",
                 "1800, 2032, 1000.0, Active, Not Active, Not Active, Not Active",
                 "garbage line"]
    s = clk.summary()
    assert s["sm_mhz"] == 2032.0 and s["sm_max_mhz"] == 2032.0 and s["samples"] == 3
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"]
    empty = bench.ClockSampler(0).summary()
    assert empty["reasons"] == ["unsampled"] and empty["samples"] == 0


def test_reference_arm_prints_the_contract_line():
    """The oracle arm on a small version of the workload: one JSON line with
    the keys the contract asks of it."""
    cmd = [sys.executable, "bench.py", "--impl", "reference", "--n", "20000", "--nq", "300",
           "--steps", "1", "--warmup", "0", "--cpu-sample", "50", "--Ls", "32", "64", "128"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1
    assert d["unit"] == "queries/s" and d["higher_is_better"] is True and d["value"] > 0
    assert d["metric"] == bench.METRIC and d["config"]["workload"] == bench.WORKLOAD
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "queries/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["L"] in (32, 64, 128) and np.isfinite(d["ms_per_step"])
