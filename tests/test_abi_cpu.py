"""The C-ABI library loads without a GPU and exports every function include/*.h
declares; host-only entry points work here (no compute calls)."""
from __future__ import annotations

import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2009_07914_gb300 import build
    build.build()
    import paper_2009_07914_gb300 as wc
    return wc.lib()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(wc[a-z0-9_]*)\s*\(", text, re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_bulk_table_calls():
    names = declared_functions()
    for want in ("wc_table_create", "wc_table_destroy", "wc_insert", "wc_retrieve", "wc_erase",
                 "wc_count_values", "wc_retrieve_multi", "wc_size", "wc_load_factor"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_plan_capacity_primes(lib):
    import sympy
    from paper_2009_07914_gb300 import api
    for n, alpha, W in [(1 << 20, 0.8, 32), (1 << 27, 0.5, 32), (1 << 27, 0.9, 32), (1 << 27, 0.99, 32),
                        (1 << 27, 0.9, 8), (1 << 28, 0.9, 4), (1000, 0.8, 4), (1, 1.0, 4), (0, 1.0, 8)]:
        want_windows = max(1, -(-int(-(-n // 1) / alpha) // W)) if n else 1
        mincap = -(-n * 1000 // int(alpha * 1000)) if n else 0
        p, c = api.wc_plan_capacity(mincap, W)
        q = max(1, -(-mincap // W))
        assert p == sympy.nextprime(q - 1) or (p == 2 and q <= 2)
        assert c == p * W and c >= mincap
        del want_windows


def test_plan_capacity_rejects_bad_arguments(lib):
    from paper_2009_07914_gb300 import api
    from paper_2009_07914_gb300._binding import WcError
    with pytest.raises(WcError):
        api.wc_plan_capacity(100, 0)
    with pytest.raises(WcError):
        api.wc_plan_capacity(1 << 40, 4)  # p would exceed 2^32


def test_status_strings(lib):
    from paper_2009_07914_gb300 import api
    assert api.wc_status_string(0) == "ok"
    assert "argument" in api.wc_status_string(1)


def test_binding_structs_match_the_c_layouts(tmp_path):
    """Every ctypes mirror of a header struct has the C struct's size and field offsets
    (a mismatch would pass garbage across the C ABI)."""
    import subprocess
    from paper_2009_07914_gb300 import _binding, roofline, serve
    pairs = [(_binding.WcTableConfig, "wc_table_config"), (_binding.WcTableInfo, "wc_table_info"),
             (_binding.WcLaunch, "wc_launch"), (_binding.WcDeviceView, "wc_device_view"),
             (roofline.WcRandAccessConfig, "wc_rand_access_config"),
             (serve.WcWork, "wc_work"), (serve.WcExecutorConfig, "wc_executor_config"),
             (serve.WcRequest, "wc_request"), (serve.WcServeConfig, "wc_serve_config"),
             (serve.WcRequestTiming, "wc_request_timing"), (serve.WcServeStats, "wc_serve_stats")]
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "wc.h"', '#include "wc_exec.h"',
             '#include "wc_serve.h"', '#include "wc_roofline.h"', "int main(void) {"]
    want = []
    for cls, cname in pairs:
        lines.append('printf("%%zu\\n", sizeof(%s));' % cname)
        want.append(ctypes.sizeof(cls))
        for f in cls._fields_:
            lines.append('printf("%%zu\\n", offsetof(%s, %s));' % (cname, f[0]))
            want.append(getattr(cls, f[0]).offset)
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    assert got == want


def test_binding_constants_match_the_header():
    """Every WC_* enumerator of include/wc.h has the same value in the Python binding."""
    from paper_2009_07914_gb300 import _binding as B
    text = open(os.path.join(ROOT, "include", "wc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    found = dict((m.group(1), int(m.group(2))) for m in re.finditer(r"\b(WC_[A-Z0-9_]+)\s*=\s*(\d+)", text))
    assert len(found) >= 25
    for name, value in found.items():
        if name == "WC_OP__N":
            continue
        assert getattr(B, name) == value, name


def test_device_api_header_compiles_for_sm103a(tmp_path):
    """The public device API (include/wc_device_api.cuh) compiles into a user's program for
    sm_103a: the example kernels of tests/device_api are built here without a GPU."""
    import shutil
    import subprocess
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path / "user_kernels.o")
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "--extended-lambda",
                        "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"), "-c",
                        os.path.join(ROOT, "tests", "device_api", "user_kernels.cu"), "-o", out],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    assert os.path.getsize(out) > 0


def test_autotune_sample_sizes_and_refusals(lib):
    """Host-side parts of the autotuner: the sample wc_table_create tunes on for
    window_width = 0 (2^20 keys for tables of up to 32 MiB of slots, else a 256 MiB table
    at load 0.9), and the argument checks that refuse a call before any device work."""
    from paper_2009_07914_gb300 import api
    assert api.wc_autotune_sample_keys(0, 4, 4, 1 << 20) == 1 << 20          # 8 MiB of 8-byte slots
    assert api.wc_autotune_sample_keys(0, 4, 4, 4 << 20) == 1 << 20          # 32 MiB: still L2-sized
    big = api.wc_autotune_sample_keys(0, 4, 4, (4 << 20) + 1)
    assert big == ((256 << 20) // 8 * 9 // 10) & ~1023 and big * 8 / 0.9 > 200 << 20
    assert api.wc_autotune_sample_keys(0, 8, 8, 1 << 30) == ((256 << 20) // 16 * 9 // 10) & ~1023
    assert api.wc_autotune_sample_keys(3, 4, 0, 1 << 30) == ((256 << 20) // 4 * 9 // 10) & ~1023
    for bad in (dict(load=1.0), dict(load=0.01), dict(sample_keys=100), dict(sample_keys=1 << 27)):
        args = dict(kind=0, key_bytes=4, value_bytes=4, load=0.9, sample_keys=1 << 14, use_cache=False, device=0)
        args.update(bad)
        with pytest.raises(Exception) as e:
            api.wc_autotune(**args)
        assert getattr(e.value, "code", None) == 1  # WC_ERR_INVALID_ARG
    for kind, kb, vb, opt in ((1, 4, 4, 0), (2, 4, 4, 0), (5, 4, 0, 0), (0, 4, 4, 2)):
        with pytest.raises(Exception) as e:
            api.wc_autotune(kind, kb, vb, load=0.9, sample_keys=1 << 14, options=opt, use_cache=False, device=0)
        assert getattr(e.value, "code", None) == 6  # WC_ERR_UNSUPPORTED
