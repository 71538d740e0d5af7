"""The benchmark's JSON line, checked on the CPU through its reference arm (the oracle timed on the host)
for every workload at small sizes: one line, the keys the line must carry, and consistent values."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

REQUIRED = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
            "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e", "impl"}


def run_bench(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                         capture_output=True, text=True, timeout=600, cwd=ROOT, check=True).stdout
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out
    return json.loads(lines[0])


@pytest.mark.parametrize("args", [
    ("--n", "256", "--lam-min", "1e-2", "--p", "1,2"),
    ("--workload", "batched", "--count", "3"),
    ("--workload", "learned", "--learned-n", "200", "--train-seqs", "1", "--test-seqs", "1", "--every", "100"),
    ("--workload", "f1", "--f1-n", "64", "--f1-iters", "3"),
])
def test_reference_line_has_the_contract_keys(args):
    d = run_bench(*args, "--steps", "2", "--warmup", "3")
    assert REQUIRED <= set(d), REQUIRED - set(d)
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 3
    assert d["higher_is_better"] is False and d["unit"] == "ms" and d["value"] > 0
    # The value is the oracle's modelled time to the step's solves; ms_per_step the measured time of one
    # benchmark step (a bounded sample of that work), so that steps x ms_per_step is the time the arm ran.
    assert 0 < d["ms_per_step"] <= d["value"] and d["data"] == "synthetic" and "workload" in d["config"]
    assert "value_model" in d
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert "l2" in d["config"]
