"""bench.py on the CPU: the reference arm (the oracle timed on host cores) prints one JSON
line in the contract's shape, and the kernel-code digest that keys the recorded DRAM
traffic ignores comments but not code."""
from __future__ import annotations

import importlib.util
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 0
    assert d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["config"]["workload"] == "sv_u32_n2^27_alpha0.90"
    cb = d["cpu_baseline"]
    # the sharded oracle on every host core, with the single-thread form beside it
    assert cb["kind"] == "oracle" and cb["cores"] == os.cpu_count() and cb["value"] == d["value"] and cb["sample"]
    assert cb["single_thread"]["cores"] == 1 and cb["single_thread"]["value"] > 0
    assert cb["host"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_kernel_digest_ignores_comments_only():
    b = _bench()
    code = "int f(int x) {\n  return x + 1;  // one more\n}\n"
    assert b._code_only(code) == b._code_only("/* header\n comment */\n" + code.replace("// one more", "// other"))
    assert b._code_only(code) != b._code_only(code.replace("x + 1", "x + 2"))
    assert len(b.source_digest()) == 16
