"""Throughput bench of the bulk hash-table hot path on GB300.

Default workload (one GPU): a single-value table of uint32 keys / uint32 values, 2^27
unique uniform random keys inserted at target load factor 0.9, then a retrieve batch of
2^27 queries (2^26 present, 2^26 absent, random order) -- the shape of the paper's
single-value experiment (Sec. V-A) at the headline density.  One step = clear the
table, bulk insert, bulk retrieve.  Inputs are resident in HBM before the timed region;
the table (1.19 GB) and the input batches (0.5-1 GB) are far larger than L2, so no flush
is needed between steps.

Prints ONE JSON line (rank 0).  `--impl reference` times the CPU oracle
(std::unordered_map) on the host instead, on a bounded sample of the same workload.
Under torchrun every rank runs an independent table on its own GPU (the path needs no
exchange between ranks: weak scaling, replicas only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import wc_inputs  # noqa: E402

SEED = 0x57C00002
METRIC = "G inserts/s & G retrievals/s at load 0.9; % of random-access HBM roofline"
# Algorithmic bytes per operation (one random 32 B sector touched per op + streamed I/O):
#   insert: 8 B of input + 1 sector read + 1 sector write = 72 B
#   retrieve: 4 B key in + 4 B value out + 1 B found mask + 1 sector read = 41 B
BYTES_PER_OP = {"insert": 72, "retrieve": 41}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="wc", choices=["wc", "reference"])
    ap.add_argument("--log2n", type=int, default=27)
    ap.add_argument("--alpha", type=float, default=0.9)
    ap.add_argument("--window", type=int, default=0)
    ap.add_argument("--group", default="0",
                    help="lanes per key: G for every operation, or G_insert,G_retrieve[,G_erase] (0 = default)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-probe", action="store_true", help="skip the random-access roofline probe")
    ap.add_argument("--kif", default="0",
                    help="sv32: keys in flight per group (1, 2; 0 = default): K for the lookups, or K_insert,K_lookup")
    ap.add_argument("--retrieve-scheme", type=int, default=0,
                    help="sv32: lookup scheme (0 = the table's, 1 direct, 2 region split, 3 grouped duplicates)")
    ap.add_argument("--alphas", default="0.5,0.8,0.9,0.95,0.99",
                    help="sv32: target loads of the density sweep reported beside the headline ('' = none)")
    ap.add_argument("--soa", action="store_true", help="sv32: struct-of-arrays table (keys and values in two arrays)")
    ap.add_argument("--no-overflow-bits", action="store_true",
                    help="sv32: table without per-window overflow bits (lookups walk to an empty slot)")
    ap.add_argument("--workload", default="sv32",
                    choices=["sv32", "sv32_small", "sv64_zipf", "mv_zipf", "mv_oa_uniform_r", "device_api", "membership",
                             "served"],
                    help="sv32 (default): 2^27 uint32 pairs at load 0.9, insert + 50%% absent retrieve; "
                         "sv32_small: 2^20 pairs at 0.8 with erase; sv64_zipf: 2^28 uint64 pairs, Zipf queries; "
                         "mv_zipf: multi-value 2^28 Zipf inserts, count + CSR retrieve; "
                         "mv_oa_uniform_r: open-addressing multi-value, 2^28 uint32 pairs with keys uniform "
                         "over 1..n/r at load 0.8, queries 1..n; "
                         "device_api: 2^27 keys produced inside one kernel and inserted / looked up per thread "
                         "with the device API, against the bulk calls on the same keys; "
                         "membership: 2^27 uint32 keys in a hash set (load 0.9), a Bloom filter (10 bits/key, k = 7) "
                         "and a counting table (Zipf keys); "
                         "served: 64 tables, Poisson requests, batched vs per-call")
    ap.add_argument("--requests", type=int, default=512, help="served: number of requests")
    ap.add_argument("--append-modes", default="1.1/1,1/r",
                    help="mv_oa_uniform_r: per-element device-API append legs into bucket tables, comma-separated "
                         "LAMBDA/S0 growth strategies ('' = none)")
    ap.add_argument("--mv-block", type=int, default=0,
                    help="mv_zipf: block size of the bucket table's insert passes (256 or 512; 0 = default)")
    ap.add_argument("--r", default="1,4,16,64", help="mv_oa_uniform_r: average copies per key, comma-separated")
    ap.add_argument("--bucket-modes", default="exact",
                    help="mv_oa_uniform_r: bucket-table legs, comma-separated: exact (one bucket of exactly each "
                         "call's count), LAMBDA/S0 (growth strategy; S0 = r for s0 = the mean values per key)")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# Sources of the single-value probe kernels (a change to any of them invalidates the
# committed traffic record of those kernels).
SV_KERNEL_SOURCES = ("wc_device.cuh", "wc_sv_kernels.cuh", "wc_sv_dispatch.cuh", "wc_partition.cuh",
                     "wc_launch.cuh", "wc_sv_p32.cu")


def _code_only(text: str) -> str:
    """C++ source without comments and blank lines (string literals with comment
    markers do not occur in these files)."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(line.rstrip() for line in text.splitlines() if line.strip())


def source_digest():
    """Digest of the code the single-value probe kernels are built from (the library's own
    sources and the public device header that holds the probing sequence), comments left
    out, so that edits of comments keep a recorded profile valid."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2009_07914_gb300", "csrc")
    paths = [os.path.join(d, name) for name in SV_KERNEL_SOURCES]
    paths.append(os.path.join(ROOT, "include", "wc_device_api.cuh"))
    for path in paths:
        with open(path, encoding="utf-8") as f:
            h.update(os.path.basename(path).encode() + _code_only(f.read()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, workload: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it was taken
    on the current kernel sources; else None."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.txt")) as f:
            lines = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    except Exception:
        return None
    for f in lines:
        if len(f) >= 4 and f[0] == kernel and f[1] == workload and f[2] == source_digest():
            return int(f[3])
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 6:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[2 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def workload(log2n: int, alpha: float):
    n = 1 << log2n
    d = wc_inputs.sv_insert_retrieve_u32(SEED, n, n // 2, n // 2)
    return n, d


def _time_oracle(o, d, n, alpha):
    """Insert then retrieve one sample into oracle object o; returns (insert_s, retrieve_s)."""
    o.reserve(int(n / alpha))
    t0 = time.perf_counter()
    o.insert(d["keys"], d["values"])
    t1 = time.perf_counter()
    o.retrieve(d["queries"])
    t2 = time.perf_counter()
    return t1 - t0, t2 - t1


def cpu_baseline(log2n_sample: int, alpha: float):
    """The oracle on the host cores, on bounded samples of the same workload (insert n
    pairs, then retrieve n queries, half absent), in its two forms: one thread over one
    std::unordered_map (reserve(n)), and sharded over every host core (one plain
    std::unordered_map per shard, key k in shard hash(k) mod T).  `value` is the sharded
    form; the single-thread one is reported beside it."""
    import oracle
    n = 1 << log2n_sample
    d = wc_inputs.sv_insert_retrieve_u32(SEED, n, n // 2, n // 2)
    ti1, tr1 = _time_oracle(oracle.SingleValue(4, 4), d, n, alpha)
    cores = os.cpu_count() or 1
    tis, trs = _time_oracle(oracle.ShardedSingleValue(4, 4, threads=cores), d, n, alpha)
    return {"value": 2 * n / (tis + trs) / 1e9, "unit": "G ops/s", "cores": cores, "kind": "oracle",
            "sample": "2^%d inserts + 2^%d retrievals (half absent), sharded std::unordered_map, one thread per "
                      "host core" % (log2n_sample, log2n_sample),
            "insert_gops": n / tis / 1e9, "retrieve_gops": n / trs / 1e9,
            "single_thread": {"value": 2 * n / (ti1 + tr1) / 1e9, "cores": 1, "insert_gops": n / ti1 / 1e9,
                              "retrieve_gops": n / tr1 / 1e9},
            "host": host_cpu()}


def host_cpu() -> dict:
    """CPU model and core count of this host (lscpu), for the CPU baseline's record."""
    model = None
    try:
        outp = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in outp.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"model": model or platform.processor() or platform.machine(), "cores": os.cpu_count()}


def random_probe(dev, table_bytes: int):
    """Live random-access ceiling of this GPU over a buffer of the table's size: the best
    rate over probe shapes (accesses in flight per thread x lanes per access) of random
    64 B reads (a probing window), 32 B reads, and 64 B read + CAS (an insert's claim)."""
    import torch
    from paper_2009_07914_gb300 import roofline as R
    nbytes = max(1 << 26, (table_bytes + 255) // 256 * 256)
    buf = torch.zeros(nbytes, dtype=torch.uint8, device=dev)
    out = {"buffer_bytes": nbytes}
    for ab, mode, key in ((64, 0, "rd64_gps"), (32, 0, "rd32_gps"), (64, 1, "rmw64_gps")):
        r = R.best_rate(buf, ab, mode, accesses=1 << 26)
        out[key] = r["accesses_per_s"] / 1e9
        out[key.replace("_gps", "_shape")] = {"in_flight": r["in_flight"], "lanes": r["lanes"]}
    # read + CAS inside one 32 MiB region (L2-resident): what the region-split insert claims in
    r = R.best_rate(buf, 64, 1, accesses=1 << 26, buffer_bytes=32 << 20)
    out["rmw64_region_gps"] = r["accesses_per_s"] / 1e9
    out["rmw64_region_shape"] = {"in_flight": r["in_flight"], "lanes": r["lanes"]}
    # the random 32 B sector rates R_rd and R_rmw over 8 GiB (HBM) and over 32 MiB (L2)
    del buf
    torch.cuda.empty_cache()
    big = torch.zeros(8 << 30, dtype=torch.uint8, device=dev)
    for mib, tag in ((8192, "8g"), (32, "l2")):
        for mode, key in ((0, "rd32"), (1, "rmw32")):
            r = R.best_rate(big, 32, mode, accesses=1 << 26, buffer_bytes=mib << 20)
            out["%s_%s_gps" % (key, tag)] = r["accesses_per_s"] / 1e9
    del big
    torch.cuda.empty_cache()
    return out


def random_bound(stream_bytes: float, window_rate_gps: float, bw_gbs: float) -> float:
    """The method's bound in G ops/s when every op streams `stream_bytes` through HBM and
    makes one random window access at the measured ceiling `window_rate_gps`:
    1 / (stream_B / BW + 1 / R_window)."""
    return 1.0 / (stream_bytes / bw_gbs + 1.0 / window_rate_gps)


def insert_launches(api, h, n: int) -> int:
    """Kernels one wc_insert launches (3 for the region-split scheme, else 1)."""
    lc = api.wc_table_get_launch(h, 0)
    info = api.wc_table_get_info(h)
    blocked = lc["scheme"] == 2 or (lc["scheme"] == 0 and info["kind"] == 0 and n >= (1 << 18)
                                     and info["table_bytes"] > (64 << 20))
    return 3 if blocked else 1


def timed(s, f):
    """Run f() between two events on stream s; returns ms."""
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s)
    f()
    b.record(s)
    b.synchronize()
    return a.elapsed_time(b)


def max_over_ranks(value: float, world: int, device) -> float:
    """The slowest rank's time: every rank runs its own table (replicas), so the job's
    time is the maximum (all_reduce MAX; no data-path collective exists)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def emit(res):
    print(json.dumps(res), flush=True)


def run_reference(args, rank, world):
    """The oracle timed on the host cores (the reference arm): every step inserts a
    2^23-pair sample of the default workload into a fresh sharded oracle (one plain
    std::unordered_map per host core) and retrieves 2^23 queries (half absent)."""
    if rank != 0:
        return
    import oracle
    steps, warm = args.steps, args.warmup
    log2s = 23
    n = 1 << log2s
    d = wc_inputs.sv_insert_retrieve_u32(SEED, n, n // 2, n // 2)
    cores = os.cpu_count() or 1
    ins, ret = [], []
    for i in range(warm + steps):
        ti, tr = _time_oracle(oracle.ShardedSingleValue(4, 4, threads=cores), d, n, args.alpha)
        if i >= warm:
            ins.append(ti)
            ret.append(tr)
    t_step = statistics.mean(a + b for a, b in zip(ins, ret))
    v = 2 * n / t_step / 1e9
    ti1, tr1 = _time_oracle(oracle.SingleValue(4, 4), d, n, args.alpha)
    sample = ("2^%d inserts + 2^%d retrievals (half absent) per step, sharded std::unordered_map, one thread per "
              "host core" % (log2s, log2s))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "G ops/s", "n_gpus": args.gpus,
        "steps": steps, "warmup": warm, "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "sv_u32_n2^%d_alpha%.2f" % (args.log2n, args.alpha), "sample_log2n": log2s},
        "cpu_baseline": {"value": v, "unit": "G ops/s", "cores": cores, "kind": "oracle", "sample": sample,
                         "single_thread": {"value": 2 * n / (ti1 + tr1) / 1e9, "cores": 1},
                         "host": host_cpu()},
        "e2e": {"value": v, "unit": "G ops/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "insert_gops": n / statistics.mean(ins) / 1e9,
        "retrieve_gops": n / statistics.mean(ret) / 1e9,
    }), flush=True)


def run_wc(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    import paper_2009_07914_gb300 as wc
    from paper_2009_07914_gb300 import api
    from paper_2009_07914_gb300.table import to_device

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    n, d = workload(args.log2n, args.alpha)
    keys = to_device(d["keys"], 4, dev)
    vals = to_device(d["values"], 4, dev)
    qk = to_device(d["queries"], 4, dev)
    out = torch.empty(n, dtype=torch.int32, device=dev)
    found = torch.empty(n, dtype=torch.uint8, device=dev)
    opts = 0 if args.no_overflow_bits else wc.WC_OPT_OVERFLOW_BITS  # half the queries are absent
    if args.soa:
        opts |= wc.WC_OPT_SOA
    h = api.wc_table_create(wc.WC_SINGLE_VALUE, 4, 4, int(np.ceil(n / args.alpha)), args.window, 0,
                            0x5EEDC0DE + rank, local_rank, options=opts)
    info = api.wc_table_get_info(h)
    tuning = None
    if args.window == 0 and not args.soa and os.environ.get("WC_AUTOTUNE", "1") != "0":
        # window_width 0: the create took the library autotuner's choice; read it back
        ns = api.wc_autotune_sample_keys(wc.WC_SINGLE_VALUE, 4, 4, int(np.ceil(n / args.alpha)), opts)
        tu = api.wc_autotune(wc.WC_SINGLE_VALUE, 4, 4, load=0.9, sample_keys=ns, options=opts, use_cache=True,
                             device=local_rank)
        tuning = {"by": "wc_autotune (window_width 0)", "sample_keys": tu["sample_keys"], "load": tu["load"],
                  "candidates": tu["candidates"], "window_width": tu["window_width"],
                  "sample_ms": [round(x, 4) for x in tu["ms"]]}
    apply_groups(api, wc, h, args.group, args.kif, args.retrieve_scheme)
    g_ins = api.wc_table_get_launch(h, wc.WC_OP_INSERT)["group_size"]
    g_ret = api.wc_table_get_launch(h, wc.WC_OP_RETRIEVE)["group_size"]
    s = torch.cuda.current_stream()

    def step(ev=None):
        if ev:
            ev[0].record(s)
        api.wc_table_clear(h, s)
        if ev:
            ev[1].record(s)
        api.wc_insert(h, keys, vals, n, s)
        if ev:
            ev[2].record(s)
        api.wc_retrieve(h, qk, out, found, n, s)
        if ev:
            ev[3].record(s)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # correctness guard on the measured configuration
    assert api.wc_size(h) == n, "insert lost keys"
    assert api.wc_get_status(h, clear=True) == 0
    nfound = int(found.sum().item())
    assert nfound == n // 2, nfound

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(s)
        for i in range(args.steps):
            step(evs[i])
        t1.record(s)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    total_ms = t0.elapsed_time(t1)
    clear_ms = [e[0].elapsed_time(e[1]) for e in evs]
    ins_ms = [e[1].elapsed_time(e[2]) for e in evs]
    ret_ms = [e[2].elapsed_time(e[3]) for e in evs]
    total_ms = max_over_ranks(total_ms, world, dev)
    ms_step = total_ms / args.steps
    value = world * 2 * n / (ms_step * 1e-3) / 1e9

    # end-to-end through the C ABI's host-buffer calls (H2D, insert, retrieve, D2H in the timed region)
    e2e = None
    if not args.no_e2e:
        hk = torch.from_numpy(d["keys"].view(np.int32)).pin_memory()
        hv = torch.from_numpy(d["values"].view(np.int32)).pin_memory()
        hq = torch.from_numpy(d["queries"].view(np.int32)).pin_memory()
        ho = torch.empty(n, dtype=torch.int32).pin_memory()
        hf = torch.empty(n, dtype=torch.uint8).pin_memory()

        def e2e_step():
            api.wc_table_clear(h, s)
            api.wc_insert_host(h, hk, hv, n, s)
            api.wc_retrieve_host(h, hq, ho, hf, n, s)
        e2e_step()
        torch.cuda.synchronize()
        assert np.array_equal(hf.numpy(), found.cpu().numpy())
        assert np.array_equal(ho.numpy()[hf.numpy() == 1], out.cpu().numpy()[hf.numpy() == 1])
        # warm-up right before the timed steps: the host-side check above leaves the GPU
        # idle for about a second, and the first step after that ran 2.5x slower
        for _ in range(max(3, args.warmup)):
            e2e_step()
        k = args.steps

        def e2e_run():
            marks = [torch.cuda.Event(enable_timing=True) for _ in range(k + 1)]
            marks[0].record(s)
            for i in range(k):
                e2e_step()
                marks[i + 1].record(s)
            torch.cuda.synchronize()
            return marks[0].elapsed_time(marks[k]) / k, [marks[i].elapsed_time(marks[i + 1]) for i in range(k)]

        e_ms, steps_ms = e2e_run()
        first = None
        # The host-memory copies share the host's memory system with whatever else runs on
        # it: a run in which one step took more than twice the median step is taken again
        # once (both runs are reported), as a clock-throttled run is.
        if max(steps_ms) > 2 * statistics.median(steps_ms):
            first = {"ms_per_step": e_ms, "step_ms": [round(x, 3) for x in steps_ms]}
            e_ms, steps_ms = e2e_run()
        per = sorted(steps_ms)
        e2e = {"value": world * 2 * n / (e_ms * 1e-3) / 1e9, "unit": "G ops/s",
               "h2d_bytes_per_step": n * 4 * 3, "d2h_bytes_per_step": n * 5, "ms_per_step": e_ms,
               "step_ms_min_median_max": [per[0], per[k // 2], per[-1]], "step_ms": [round(x, 3) for x in steps_ms],
               "calls": "wc_insert_host + wc_retrieve_host from pinned buffers (chunked copies on the "
                        "table's copy streams, overlapping the kernels)"}
        if first is not None:
            e2e["first_run_stalled"] = first

    if rank != 0:
        return
    peak, peak_kind = peaks()
    ins, ret = statistics.median(ins_ms), statistics.median(ret_ms)
    dom = "insert" if ins >= ret else "retrieve"
    dom_ms = max(ins, ret)
    achieved = BYTES_PER_OP[dom] * n / (dom_ms * 1e-3) / 1e9
    workload_name = "sv_u32_n2^%d_alpha%.2f" % (args.log2n, args.alpha)
    kif_ret = api.wc_table_get_launch(h, wc.WC_OP_RETRIEVE)["keys_in_flight"]
    kname = "k_sv_insert" if dom == "insert" else ("k_sv_retrieve2" if kif_ret == 2 else "k_sv_retrieve")
    traffic = ncu_traffic(kname, workload_name)
    cpu = None if args.no_cpu else cpu_baseline(23, args.alpha)
    res = {
        "metric": METRIC, "value": value, "unit": "G ops/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": workload_name, "n": n, "queries": n, "present_fraction": 0.5,
                   "capacity": info["capacity"], "achieved_alpha": n / info["capacity"],
                   "window_slots": info["window_width"], "tuning": tuning, "group_insert": g_ins,
                   "group_retrieve": g_ret,
                   "insert_keys_in_flight": api.wc_table_get_launch(h, wc.WC_OP_INSERT)["keys_in_flight"],
                   "retrieve_keys_in_flight": api.wc_table_get_launch(h, wc.WC_OP_RETRIEVE)["keys_in_flight"],
                   "retrieve_scheme": {0: "auto (direct)", 1: "direct", 2: "region split", 3: "grouped duplicates"}[
                       api.wc_table_get_launch(h, wc.WC_OP_RETRIEVE)["scheme"]],
                   "table_bytes": info["table_bytes"], "overflow_bits": bool(info["options"] & 1),
                   "layout": "struct of arrays" if info["options"] & 2 else "packed 64-bit slots",
                   "l2": "no flush: inputs and table larger than L2 (table %.2f GB, keys %.2f GB)"
                         % (info["table_bytes"] / 1e9, n * 4 / 1e9),
                   "parallelism": "replicas (independent table per GPU)"},
        "insert_gops": n / (ins * 1e-3) / 1e9, "retrieve_gops": n / (ret * 1e-3) / 1e9,
        "clear_ms": statistics.median(clear_ms), "insert_ms": ins, "retrieve_ms": ret,
        "insert_ms_mean": statistics.mean(ins_ms), "retrieve_ms_mean": statistics.mean(ret_ms),
        "roofline": {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind,
                     "bytes_per_op": BYTES_PER_OP[dom], "traffic": traffic,
                     # the DRAM bytes the kernel actually moves (recorded ncu traffic) over its
                     # measured duration: how close the random walk runs to the copy bandwidth
                     "dram_gbs": None if traffic is None else traffic / (dom_ms * 1e-3) / 1e9,
                     "dram_frac": None if traffic is None else traffic / (dom_ms * 1e-3) / 1e9 / peak,
                     "dram_sectors_per_op": None if traffic is None else traffic / 32 / n,
                     # a random miss fills a whole 128-byte L2 line (measured with the library's
                     # random-access probe): the traffic in lines per operation
                     "dram_lines_per_op": None if traffic is None else traffic / 128 / n},
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": (insert_launches(api, h, n) + 1) * args.steps,
        "clocks": clk.summary(),
    }
    if args.alphas:
        res["load_sweep"] = load_sweep(args, api, wc, h, keys, vals, qk, out, found, n, s, peak, rank, local_rank)
    if not args.no_probe:
        pr = random_probe(dev, info["table_bytes"])
        # retrieve reads ~1 window of W slots per present key and a few per absent key;
        # report the query rate against the random-window read rate of the same buffer
        ret_bound = random_bound(9, pr["rd64_gps"], peak)
        ins_bound = random_bound(8, pr["rmw64_gps"], peak)
        # the region-split insert: streamed passes (histogram 4 B, split 8 B in + 8 B out,
        # sweep 8 B in per pair) and the table read and written back once, region by region,
        # plus one read + CAS per pair inside an L2-resident region
        tbl = 2 * info["table_bytes"] / n
        split_bound = random_bound(28 + tbl, pr["rmw64_region_gps"], peak)
        res["random_roofline"] = dict(pr, retrieve_bound_gops=ret_bound, insert_bound_gops=ins_bound,
                                      retrieve_frac_of_rd64=res["retrieve_gops"] / pr["rd64_gps"],
                                      insert_frac_of_rmw64=res["insert_gops"] / pr["rmw64_gps"],
                                      retrieve_frac_of_bound=res["retrieve_gops"] / ret_bound,
                                      insert_frac_of_bound=res["insert_gops"] / ins_bound,
                                      theoretical_sector_gps=peak / 32,
                                      retrieve_frac_of_theoretical_sectors=res["retrieve_gops"] / (peak / 32),
                                      insert_frac_of_theoretical_sectors=2 * res["insert_gops"] / (peak / 32),
                                      retrieve_frac_of_rd32_8g=res["retrieve_gops"] / pr["rd32_8g_gps"],
                                      insert_frac_of_rmw32_8g=res["insert_gops"] / pr["rmw32_8g_gps"],
                                      insert_region_split_bound_gops=split_bound,
                                      insert_frac_of_region_split_bound=res["insert_gops"] / split_bound,
                                      formula="1 / (stream_B / BW + 1 / R_window): retrieve 9 B streamed + one 64 B "
                                              "random read; insert 8 B + one 64 B random read + CAS; region-split "
                                              "insert 28 B + 2 x table bytes per pair streamed + one 64 B read + CAS "
                                              "in a 32 MiB region")
    print(json.dumps(res), flush=True)
    api.wc_table_destroy(h)


def apply_groups(api, wc, h, spec: str, kif: str = "0", retrieve_scheme: int = 0):
    """--group: one lane count for every operation, or one per operation (insert,
    retrieve[, erase]); 0 keeps the table's default.  kif: keys in flight per group, for
    the lookups alone ("2") or for insert and lookups ("2,2"); 0 keeps the default.
    retrieve_scheme: the lookups' WC_SCHEME_* (0 keeps the default)."""
    gs = [int(x) for x in str(spec).split(",") if x.strip()]
    if len(gs) == 1:
        gs = gs * 3
    for op, g in zip((wc.WC_OP_INSERT, wc.WC_OP_RETRIEVE, wc.WC_OP_ERASE), gs):
        if g:
            lc = api.wc_table_get_launch(h, op)
            api.wc_table_set_launch(h, op, g, lc["block_threads"], lc["blocks_per_sm"], lc["scheme"], lc["region_mib"],
                                    lc["keys_in_flight"])
    ks = [int(x) for x in str(kif).split(",") if x.strip()]
    ops = (wc.WC_OP_RETRIEVE,) if len(ks) == 1 else (wc.WC_OP_INSERT, wc.WC_OP_RETRIEVE)
    for op, k in zip(ops, ks):
        if k:
            lc = api.wc_table_get_launch(h, op)
            api.wc_table_set_launch(h, op, lc["group_size"], lc["block_threads"], lc["blocks_per_sm"], lc["scheme"],
                                    lc["region_mib"], k)
    if retrieve_scheme:
        lc = api.wc_table_get_launch(h, wc.WC_OP_RETRIEVE)
        api.wc_table_set_launch(h, wc.WC_OP_RETRIEVE, lc["group_size"], lc["block_threads"], lc["blocks_per_sm"],
                                retrieve_scheme, lc["region_mib"], lc["keys_in_flight"])


def load_sweep(args, api, wc, h_main, keys, vals, qk, out, found, n, s, peak, rank, local_rank):
    """The paper's density sweep (Sec. V-A) on the default workload: for every target load
    of --alphas, a table of the bench's kind (same options and shapes as the headline
    table) is filled with the 2^27 pairs and queried with the 2^27 half-absent queries;
    insert and retrieve are timed separately with CUDA events (median of the steps), and
    every table is checked (size, no status flag, found count) before it is timed."""
    import torch
    info_main = api.wc_table_get_info(h_main)
    rows = []
    steps = max(3, min(args.steps, 10))
    for a in (float(x) for x in args.alphas.split(",") if x.strip()):
        h = api.wc_table_create(wc.WC_SINGLE_VALUE, 4, 4, int(np.ceil(n / a)), args.window, 0, 0x5EEDC0DE + rank,
                                local_rank, options=info_main["options"])
        apply_groups(api, wc, h, args.group, args.kif, args.retrieve_scheme)
        info = api.wc_table_get_info(h)
        ins, ret = [], []
        for i in range(2 + steps):
            api.wc_table_clear(h, s)
            ti = timed(s, lambda: api.wc_insert(h, keys, vals, n, s))
            tr = timed(s, lambda: api.wc_retrieve(h, qk, out, found, n, s))
            if i == 0:
                assert api.wc_size(h) == n and api.wc_get_status(h, clear=True) == 0, a
                assert int(found.sum().item()) == n // 2, a
            if i >= 2:
                ins.append(ti)
                ret.append(tr)
        im, rm = statistics.median(ins), statistics.median(ret)
        rows.append({"target_alpha": a, "achieved_alpha": n / info["capacity"], "capacity": info["capacity"],
                     "insert_gops": n / (im * 1e-3) / 1e9, "retrieve_gops": n / (rm * 1e-3) / 1e9,
                     "insert_ms": im, "retrieve_ms": rm,
                     "insert_frac": BYTES_PER_OP["insert"] * n / (im * 1e-3) / 1e9 / peak,
                     "retrieve_frac": BYTES_PER_OP["retrieve"] * n / (rm * 1e-3) / 1e9 / peak})
        api.wc_table_destroy(h)
    torch.cuda.synchronize()
    return rows


def _common(args, workload_name, metric, value, unit, ms_step, dtype, config, clk, launches, extra):
    res = {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
           "data": "synthetic", "config": dict(config, workload=workload_name), "gpu_launches": launches,
           "clocks": clk.summary()}
    res.update(extra)
    emit(res)


def run_sv32_small(args, dev):
    """2^20 unique uint32 pairs at load 0.8 (a 10 MB table that fits in L2): insert, retrieve
    2^20 present + 2^20 absent, erase a random half, retrieve all 2^21 again; with and
    without the L2 access-policy window on the slot array."""
    import torch
    from paper_2009_07914_gb300 import api
    from paper_2009_07914_gb300.table import to_device
    n = 1 << 20
    d = wc_inputs.sv_insert_retrieve_u32(0x57C00001, n, n, n)
    keys, vals, qk = (to_device(d[k], 4, dev) for k in ("keys", "values", "queries"))
    drop = to_device(d["keys"][wc_inputs.shuffle_index(0x57C00001, n)[: n // 2]], 4, dev)
    out = torch.empty(2 * n, dtype=torch.int32, device=dev)
    found = torch.empty(2 * n, dtype=torch.uint8, device=dev)
    s = torch.cuda.current_stream()
    results = {}
    for persist in (False, True):
        h = api.wc_table_create(0, 4, 4, int(np.ceil(n / 0.8)), args.window, 0, 0x5EEDC0DE, dev.index, persist)

        def step():
            api.wc_table_clear(h, s)
            api.wc_insert(h, keys, vals, n, s)
            api.wc_retrieve(h, qk, out, found, 2 * n, s)
            api.wc_erase(h, drop, n // 2, s)
            api.wc_retrieve(h, qk, out, found, 2 * n, s)
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        assert api.wc_size(h) == n - n // 2 and int(found.sum()) == n - n // 2
        with ClockSampler(dev.index) as clk:
            ms = timed(s, lambda: [step() for _ in range(args.steps)]) / args.steps
        results[persist] = ms
        info = api.wc_table_get_info(h)
        api.wc_table_destroy(h)
    ops = n + 2 * n + n // 2 + 2 * n
    best = min(results.values())
    _common(args, "sv_u32_n2^20_alpha0.80_erase", "G ops/s (insert + retrieve + erase + retrieve)", ops / best / 1e6,
            "G ops/s", best, "u32", {"n": n, "capacity": info["capacity"], "table_bytes": info["table_bytes"],
                                     "l2": "table fits in L2"}, clk, 4 * args.steps,
            {"ms_per_step_no_l2_window": results[False], "ms_per_step_l2_window": results[True]})


def run_sv64_zipf(args, dev):
    """2^28 unique uint64 pairs at load 0.9 (4.8 GB of 16-byte slots, one 128-bit CAS per
    claim); 2^28 queries drawn Zipf(1.1) over the inserted keys."""
    import torch
    from paper_2009_07914_gb300 import api
    from paper_2009_07914_gb300.table import to_device
    log2n = min(args.log2n, 28) if args.log2n != 27 else 28
    n = 1 << log2n
    d = wc_inputs.sv_u64_zipf(0x57C00003, n, n)
    keys, vals, qk = (to_device(d[k], 8, dev) for k in ("keys", "values", "queries"))
    out = torch.empty(n, dtype=torch.int64, device=dev)
    found = torch.empty(n, dtype=torch.uint8, device=dev)
    s = torch.cuda.current_stream()
    h = api.wc_table_create(0, 8, 8, int(np.ceil(n / 0.9)), args.window, 0, 0x5EEDC0DE, dev.index)
    info = api.wc_table_get_info(h)
    import paper_2009_07914_gb300 as wc
    apply_groups(api, wc, h, args.group, args.kif, args.retrieve_scheme)
    ev = []

    def step(rec):
        api.wc_table_clear(h, s)
        t0 = timed(s, lambda: api.wc_insert(h, keys, vals, n, s))
        t1 = timed(s, lambda: api.wc_retrieve(h, qk, out, found, n, s))
        if rec:
            ev.append((t0, t1))
    for _ in range(args.warmup):
        step(False)
    assert api.wc_size(h) == n and int(found.sum()) == n
    with ClockSampler(dev.index) as clk:
        for _ in range(args.steps):
            step(True)
    ins = statistics.median(e[0] for e in ev)
    ret = statistics.median(e[1] for e in ev)
    # the same lookups with equal queries of each warp block probed once (WC_SCHEME_DEDUP)
    import paper_2009_07914_gb300 as wc
    lc = api.wc_table_get_launch(h, wc.WC_OP_RETRIEVE)
    direct_out = out.clone()
    api.wc_table_set_launch(h, wc.WC_OP_RETRIEVE, lc["group_size"], lc["block_threads"], lc["blocks_per_sm"],
                            scheme=wc.WC_SCHEME_DEDUP)
    dd = [timed(s, lambda: api.wc_retrieve(h, qk, out, found, n, s)) for _ in range(args.warmup + args.steps)]
    assert torch.equal(out, direct_out) and int(found.sum()) == n
    ret_dedup = statistics.median(dd[args.warmup:])
    api.wc_table_set_launch(h, wc.WC_OP_RETRIEVE, lc["group_size"], lc["block_threads"], lc["blocks_per_sm"],
                            scheme=lc["scheme"])
    peak, kind = peaks()
    _common(args, "sv_u64_n2^%d_alpha0.90_zipf1.1" % log2n, "G ops/s (insert + Zipf retrieve)",
            2 * n / ((ins + ret) * 1e-3) / 1e9, "G ops/s", ins + ret, "u64",
            {"n": n, "capacity": info["capacity"], "table_bytes": info["table_bytes"],
             "window_slots": info["window_width"], "launch": {
                 op: {k: lc_[k] for k in ("group_size", "keys_in_flight", "scheme")}
                 for op, lc_ in (("insert", api.wc_table_get_launch(h, wc.WC_OP_INSERT)), ("retrieve", lc))},
             "l2": "no flush: table 4.8 GB"}, clk,
            (insert_launches(api, h, n) + 1) * args.steps,
            {"insert_gops": n / ins / 1e6, "retrieve_gops": n / ret / 1e6, "insert_ms": ins, "retrieve_ms": ret,
             "retrieve_dedup_gops": n / ret_dedup / 1e6, "retrieve_dedup_ms": ret_dedup,
             "roofline": {"bound": "hbm", "kernel": "k_sv_retrieve", "achieved": 48 * n / (ret * 1e-3) / 1e9,
                          "peak": peak, "unit": "GB/s", "frac": 48 * n / (ret * 1e-3) / 1e9 / peak,
                          "bytes_per_op": 48, "traffic": None}})
    api.wc_table_destroy(h)


def run_mv_zipf(args, dev):
    """Multi-value: 2^28 inserts whose uint64 keys are drawn Zipf(1.1) over 2^24 distinct
    keys (value = insert index, uint32); count_values then retrieve_multi for the whole
    universe plus 2^22 absent keys, into CSR offsets."""
    import torch
    from paper_2009_07914_gb300 import api
    from paper_2009_07914_gb300.table import to_device
    log2n = 28 if args.log2n == 27 else args.log2n  # default: 2^28 inserts over 2^24 keys
    uni, n, na = 1 << (log2n - 4), 1 << log2n, 1 << (log2n - 6)
    d = wc_inputs.mv_zipf_u64(0x57C00004, uni, n, na)
    keys = to_device(d["keys"], 8, dev)
    vals = to_device(d["values"], 4, dev)
    q = to_device(d["queries"], 8, dev)
    nq = q.numel()
    offs = torch.empty(nq + 1, dtype=torch.int64, device=dev)
    out = torch.empty(n, dtype=torch.int32, device=dev)
    s = torch.cuda.current_stream()
    h = api.wc_table_create(1, 8, 4, int(np.ceil(uni / 0.8)), args.window, n + (n >> 3), 0x5EEDC0DE, dev.index)
    if args.mv_block:
        lc = api.wc_table_get_launch(h, 0)
        api.wc_table_set_launch(h, 0, lc["group_size"], args.mv_block, lc["blocks_per_sm"], lc["scheme"],
                                lc["region_mib"])
    info = api.wc_table_get_info(h)
    ev = []

    def step(rec):
        api.wc_table_clear(h, s)
        t0 = timed(s, lambda: api.wc_insert(h, keys, vals, n, s))
        t1 = timed(s, lambda: api.wc_count_values(h, q, offs, nq, want_total=False, stream=s))
        t2 = timed(s, lambda: api.wc_retrieve_multi(h, q, offs, out, nq, s))
        if rec:
            ev.append((t0, t1, t2))
    for _ in range(args.warmup):
        step(False)
    assert api.wc_size(h) == n and int(offs[-1].item()) == n and api.wc_get_status(h, True) == 0
    with ClockSampler(dev.index) as clk:
        for _ in range(args.steps):
            step(True)
    ins, cnt, ret = (statistics.median(e[i] for e in ev) for i in range(3))
    total = ins + cnt + ret
    _common(args, "mv_u64u32_n2^%d_zipf1.1_over2^%d" % (log2n, log2n - 4),
            "G ops/s (inserts + queries + values retrieved)",
            (n + nq + n) / (total * 1e-3) / 1e9, "G ops/s", total, "u64/u32",
            {"n_inserts": n, "universe": uni, "queries": nq, "key_store_capacity": info["capacity"],
             "insert_block": api.wc_table_get_launch(h, 0)["block_threads"],
             "pool": info["pool_capacity"], "l2": "no flush: 2 GB of inserts, 1 GB pool"}, clk,
            10 * args.steps,  # hist, scatter, count, alloc, scatter; count, 3 scan kernels; gather
            {"insert_gops": n / ins / 1e6, "count_gqps": nq / cnt / 1e6, "retrieve_multi_gvals": n / ret / 1e6,
             "insert_ms": ins, "count_ms": cnt, "retrieve_multi_ms": ret, "distinct_keys": api.wc_num_keys(h)})
    api.wc_table_destroy(h)


def run_mv_oa_uniform_r(args, dev):
    """The paper's multi-value workload (Sec. V-C): n uint32 keys drawn uniformly from
    1..n/r (value = insert index), then count_values + retrieve_multi for all of 1..n, so
    exactly n values come back.  For every r of --r, both multi-value layouts: the
    open-addressing table (one slot per pair, load 0.8 over the pairs) and the key-once
    bucket table (key store at load 0.8 over the n/r keys, exact-size buckets).  One step
    = clear + insert + count + retrieve on one table; the value is the open-addressing
    table's throughput over every r, the bucket table's is reported beside it."""
    import torch
    from paper_2009_07914_gb300 import WC_OP_COUNT, WC_OP_INSERT, WC_OP_RETRIEVE, api
    from paper_2009_07914_gb300.table import to_device
    log2n = 28 if args.log2n == 27 else args.log2n
    n = 1 << log2n
    rs = [int(x) for x in args.r.split(",")]
    q = to_device(np.arange(1, n + 1, dtype=np.uint32), 4, dev)
    vals = to_device(np.arange(n, dtype=np.uint32), 4, dev)
    offs = torch.empty(n + 1, dtype=torch.int64, device=dev)
    out = torch.empty(n, dtype=torch.int32, device=dev)
    s = torch.cuda.current_stream()
    h = api.wc_table_create(2, 4, 4, int(np.ceil(n / 0.8)), args.window, 0, 0x5EEDC0DE, dev.index)
    if int(args.group.split(",")[0]):
        for op in (WC_OP_INSERT, WC_OP_RETRIEVE, WC_OP_COUNT):
            api.wc_table_set_launch(h, op, int(args.group.split(",")[0]), 256, 0, 0, 0)
    info = api.wc_table_get_info(h)
    modes = [m.strip() for m in args.bucket_modes.split(",") if m.strip()]
    amodes = [m.strip() for m in args.append_modes.split(",") if m.strip()]
    res = {"oa": {}}
    for m in modes:
        res["bucket" if m == "exact" else "bucket_" + m] = {}
    for m in amodes:
        res["append_" + m] = {}

    def growth_of(m, r):
        lam_s, s0_s = m.split("/")
        return float(lam_s), (r if s0_s == "r" else int(s0_s))
    launches = 0
    with ClockSampler(dev.index) as clk:
        for r in rs:
            keys = to_device(wc_inputs.mv_uniform_r(0x57C00005 + r, n, r)["keys"].astype(np.uint32), 4, dev)
            legs = [("oa", h)]
            for m in modes:
                if m == "exact":
                    s0, lam = 0, 1.0
                else:
                    lam, s0 = growth_of(m, r)
                # pool: values + headers + padding of the largest layout (s0 = 1, lambda = 1: 4 per value)
                pool = n + 2 * (n // r) + 1024 if s0 == 0 else 4 * n + 1024
                legs.append(("bucket" if m == "exact" else "bucket_" + m,
                             api.wc_table_create(1, 4, 4, int(np.ceil(max(1, n // r) / 0.8)), 0, pool, 0x5EEDC0DE,
                                                 dev.index, bucket_first_size=s0, bucket_growth=lam)))
            for m in amodes:  # the same tables, filled by per-element device-API appends
                lam, s0 = growth_of(m, r)
                legs.append(("append_" + m,
                             api.wc_table_create(1, 4, 4, int(np.ceil(max(1, n // r) / 0.8)), 0, 4 * n + 1024,
                                                 0x5EEDC0DE, dev.index, bucket_first_size=s0, bucket_growth=lam)))
            from paper_2009_07914_gb300.roofline import wc_bench_mv_append
            for name, t in legs:
                ev = []
                ins = (lambda: wc_bench_mv_append(t, keys, vals, n, s)) if name.startswith("append_") else \
                    (lambda: api.wc_insert(t, keys, vals, n, s))
                for i in range(args.warmup + args.steps):
                    api.wc_table_clear(t, s)
                    t0 = timed(s, ins)
                    t1 = timed(s, lambda: api.wc_count_values(t, q, offs, n, want_total=False, stream=s))
                    t2 = timed(s, lambda: api.wc_retrieve_multi(t, q, offs, out, n, s))
                    if i >= args.warmup:
                        ev.append((t0, t1, t2))
                    if i == 0:
                        assert api.wc_size(t) == n and int(offs[-1].item()) == n and api.wc_get_status(t, True) == 0
                ins, cnt, ret = (statistics.median(e[j] for e in ev) for j in range(3))
                res[name][str(r)] = {"insert_gops": n / ins / 1e6, "retrieve_gqps": n / (cnt + ret) / 1e6,
                                     "count_gqps": n / cnt / 1e6, "insert_ms": ins, "count_ms": cnt,
                                     "retrieve_multi_ms": ret}
                if name != "oa":
                    res[name][str(r)]["pool_elements_per_value"] = api.wc_value_pool_used(t) / n
                # OA: hist + scatter + insert, walk + 3 scan kernels, walk; bucket: hist +
                # scatter + count + alloc + scatter, count + 3 scan kernels, gather
                # append legs: one append kernel, count + 3 scan kernels, gather
                launches += (8 if name == "oa" else 6 if name.startswith("append_") else 10) * args.steps
            for name, t in legs[1:]:
                api.wc_table_destroy(t)
            del keys
    total = {m: sum(v["insert_ms"] + v["count_ms"] + v["retrieve_multi_ms"] for v in res[m].values()) for m in res}
    _common(args, "mv_oa_u32_n2^%d_uniform_r%s_alpha0.80" % (log2n, "-".join(map(str, rs))),
            "G ops/s (inserts + queries, over every r)", 2 * n * len(rs) / (total["oa"] * 1e-3) / 1e9, "G ops/s",
            total["oa"], "u32", {"n": n, "r": rs, "capacity": info["capacity"], "table_bytes": info["table_bytes"],
                                 "window_slots": info["window_width"],
                                 "groups": {op: api.wc_table_get_launch(h, c)["group_size"] for op, c in
                                            (("insert", WC_OP_INSERT), ("count", WC_OP_COUNT),
                                             ("retrieve_multi", WC_OP_RETRIEVE))},
                                 "l2": "no flush: 2.7 GB table, 1 GB inputs"}, clk, launches,
            dict({"per_r": res["oa"]},
                 **{k + "_per_r": v for k, v in res.items() if k != "oa"},
                 **{k + "_value": 2 * n * len(rs) / (total[k] * 1e-3) / 1e9 for k in res if k != "oa"}))
    api.wc_table_destroy(h)


def run_device_api(args, dev):
    """Device-side API (fused producer): one kernel whose threads produce the keys
    k_i = (i * 2654435761 mod 2^32) xor seed (distinct) and insert (k_i, i), then one whose
    threads look k_i up; against the bulk insert and retrieve of the same keys held in
    device memory.  2^27 keys into a table at load 0.9 with overflow bits."""
    import torch

    import paper_2009_07914_gb300 as wc
    from paper_2009_07914_gb300 import api
    from paper_2009_07914_gb300.roofline import wc_bench_device_api, wc_bench_device_api_group
    from paper_2009_07914_gb300.table import to_device
    n = 1 << args.log2n
    seed = 0x2468ACE1
    idx = np.arange(n, dtype=np.uint64)
    k = ((idx * np.uint64(2654435761)) & np.uint64(0xFFFFFFFF)).astype(np.uint32) ^ np.uint32(seed)
    valid = (k != 0) & (k != 0xFFFFFFFF)
    nv = int(valid.sum())
    keys, vals = to_device(k, 4, dev), to_device(idx.astype(np.uint32), 4, dev)
    out = torch.empty(n, dtype=torch.int32, device=dev)
    found = torch.empty(n, dtype=torch.uint8, device=dev)
    sink = torch.zeros(1, dtype=torch.int64, device=dev)
    want = int(idx[valid].astype(np.uint64).sum(dtype=np.uint64) & np.uint64(0x7FFFFFFFFFFFFFFF))
    h = api.wc_table_create(0, 4, 4, int(np.ceil(n / args.alpha)), args.window, 0, 0x5EEDC0DE, dev.index,
                            options=0 if args.no_overflow_bits else wc.WC_OPT_OVERFLOW_BITS)
    s = torch.cuda.current_stream()
    ev = []
    with ClockSampler(dev.index) as clk:
        for i in range(args.warmup + args.steps):
            api.wc_table_clear(h, s)
            sink.zero_()
            t0 = timed(s, lambda: wc_bench_device_api(h, 0, n, seed, None, s))
            t1 = timed(s, lambda: wc_bench_device_api(h, 1, n, seed, sink, s))
            if i == 0:
                assert api.wc_size(h) == nv and int(sink.item()) & 0x7FFFFFFFFFFFFFFF == want
            api.wc_table_clear(h, s)
            t2 = timed(s, lambda: api.wc_insert(h, keys, vals, n, s))
            t3 = timed(s, lambda: api.wc_retrieve(h, keys, out, found, n, s))
            if i == 0:
                assert api.wc_size(h) == nv and int(found.sum()) == nv
            if i >= args.warmup:
                ev.append((t0, t1, t2, t3))
    # the group-cooperative forms: tiles of G threads per key
    grp = {}
    for G in (2, 4):
        gev = []
        for i in range(args.warmup + args.steps):
            api.wc_table_clear(h, s)
            sink.zero_()
            t0 = timed(s, lambda: wc_bench_device_api_group(h, 0, G, n, seed, None, s))
            t1 = timed(s, lambda: wc_bench_device_api_group(h, 1, G, n, seed, sink, s))
            if i == 0:
                assert api.wc_size(h) == nv and int(sink.item()) & 0x7FFFFFFFFFFFFFFF == want
            if i >= args.warmup:
                gev.append((t0, t1))
        gi, gl = (statistics.median(e[j] for e in gev) for j in range(2))
        grp["group%d_insert_gops" % G] = n / gi / 1e6
        grp["group%d_lookup_gops" % G] = n / gl / 1e6
    fi, fl, bi, br = (statistics.median(e[j] for e in ev) for j in range(4))
    _common(args, "device_api_u32_n2^%d_alpha%.2f" % (args.log2n, args.alpha),
            "G ops/s (device-API fused insert + lookup)", 2 * n / ((fi + fl) * 1e-3) / 1e9, "G ops/s", fi + fl, "u32",
            {"n": n, "keys": "produced in the kernel: (i * 2654435761 mod 2^32) xor seed",
             "overflow_bits": not args.no_overflow_bits,
             "l2": "no flush: table 1.19 GB"}, clk, 2 * args.steps,
            {"fused_insert_gops": n / fi / 1e6, "fused_lookup_gops": n / fl / 1e6,
             "bulk_insert_gops": n / bi / 1e6, "bulk_retrieve_gops": n / br / 1e6,
             "fused_insert_ms": fi, "fused_lookup_ms": fl, "bulk_insert_ms": bi, "bulk_retrieve_ms": br, **grp})
    api.wc_table_destroy(h)


def run_membership(args, dev):
    """The other table types of Sec. IV on 2^27 uint32 keys: a hash set at load 0.9 (insert,
    then membership of the keys plus as many absent ones), a blocked Bloom filter with 10
    bits per key and k = 7 (insert, membership, measured false-positive rate), and a
    counting table fed 2^27 Zipf(1.1) draws over 2^24 keys (insert, count lookups)."""
    import torch

    import paper_2009_07914_gb300 as wc
    from paper_2009_07914_gb300 import api
    from paper_2009_07914_gb300.table import to_device
    n = 1 << args.log2n
    d = wc_inputs.sv_insert_retrieve_u32(0x57C00006, n, n // 2, n // 2)
    keys, q = to_device(d["keys"], 4, dev), to_device(d["queries"], 4, dev)
    pres = torch.from_numpy((d["q_src"] >= 0).astype(np.uint8)).to(dev)
    found = torch.empty(n, dtype=torch.uint8, device=dev)
    z = wc_inputs.mv_zipf_u64(0x57C00007, 1 << 24, n, 1 << 20)
    zk = to_device(((z["keys"] & np.uint64(0x7FFFFFFF)) | np.uint64(1)).astype(np.uint32), 4, dev)
    zq = to_device(((z["queries"] & np.uint64(0x7FFFFFFF)) | np.uint64(1)).astype(np.uint32), 4, dev)
    counts = torch.empty(zq.numel(), dtype=torch.int32, device=dev)
    cfound = torch.empty(zq.numel(), dtype=torch.uint8, device=dev)
    s = torch.cuda.current_stream()
    hs = api.wc_table_create(wc.WC_HASH_SET, 4, 0, int(np.ceil(n / 0.9)), 0, 0, 0x5EEDC0DE, dev.index,
                             options=wc.WC_OPT_OVERFLOW_BITS)
    bf = api.wc_table_create(wc.WC_BLOOM_FILTER, 4, 0, 10 * n, 7, 0, 0x5EEDC0DE, dev.index)
    ct = api.wc_table_create(wc.WC_COUNTING, 4, 4, int(np.ceil((1 << 24) / 0.9)), 0, 0, 0x5EEDC0DE, dev.index)
    ev = []
    with ClockSampler(dev.index) as clk:
        for i in range(args.warmup + args.steps):
            r = []
            for h, ins_keys, ins_n, qk, qn, out in ((hs, keys, n, q, n, None), (bf, keys, n, q, n, None),
                                                    (ct, zk, n, zq, zq.numel(), counts)):
                api.wc_table_clear(h, s)
                r.append(timed(s, lambda: api.wc_insert(h, ins_keys, None, ins_n, s)))
                if out is None:
                    r.append(timed(s, lambda: api.wc_contains(h, qk, found, qn, s)))
                else:
                    r.append(timed(s, lambda: api.wc_retrieve(h, qk, out, cfound, qn, s)))
                if i == 0 and h == hs:
                    assert torch.equal(found, pres) and api.wc_size(hs) == n
                if i == 0 and h == bf:
                    fpos = int((found & (1 - pres)).sum().item()) / int((1 - pres).sum().item())
                    assert bool((found >= pres).all())  # no false negatives
            if i >= args.warmup:
                ev.append(r)
    med = [statistics.median(e[j] for e in ev) for j in range(6)]
    nz = zq.numel()
    total = sum(med)
    _common(args, "membership_u32_n2^%d" % args.log2n, "G ops/s (set + Bloom + counting: inserts + lookups)",
            (4 * n + n + nz) / (total * 1e-3) / 1e9, "G ops/s", total, "u32",
            {"n": n, "set_alpha": 0.9, "bloom_bits_per_key": 10, "bloom_k": 7,
             "counting": "2^27 Zipf(1.1) draws over 2^24 keys", "l2": "no flush: tables and inputs > L2"}, clk,
            6 * args.steps,
            {"set_insert_gops": n / med[0] / 1e6, "set_contains_gops": n / med[1] / 1e6,
             "bloom_insert_gops": n / med[2] / 1e6, "bloom_contains_gops": n / med[3] / 1e6,
             "bloom_false_positive_rate": fpos, "counting_insert_gops": n / med[4] / 1e6,
             "counting_lookup_gops": nz / med[5] / 1e6})
    for h in (hs, bf, ct):
        api.wc_table_destroy(h)


def run_served(args, dev):
    """64 uint32 tables (capacity 2^U(16,26), pre-filled to load U(0,0.6)); Poisson
    requests with batch sizes 2^U(log2 1000, 24), 60/35/5 insert/retrieve/erase.  Each
    mode serves the same trace from the same start: per-call launches and batched
    (continuous batching into the persistent executor, up to 2^26 keys per launch), closed
    loop and at 0.5/0.8/0.95 of the per-call saturation rate; p50/p99 latency per run.
    One more closed-loop run caps batches at 2^22 keys and sends requests of 2^20 keys
    or more as their own bulk call."""
    import torch
    from paper_2009_07914_gb300 import serve
    tr = wc_inputs.serving_trace(0x57C00005, n_tables=64, n_requests=args.requests)
    dt = serve.DeviceTrace(tr, device=dev.index, window_width=8)
    from paper_2009_07914_gb300 import tune
    groups = tune.executor_groups(8, use_cache=False)  # lanes per key of the executor, timed on this GPU
    ex = serve.wc_executor_create(dev.index, 8, max_items=1024, tile_keys=4096, **groups)
    nreq = len(tr["requests"])
    keys_total = sum(r["keys"].size for r in tr["requests"])
    from paper_2009_07914_gb300 import api
    dt.reset()  # the pre-fill grows the tables' scratch to its size for the run
    resident = sum(i["device_bytes"] + i["work_bytes"] for i in map(api.wc_table_get_info, dt.tables))
    # the tables plus 512 MiB of request buffers: admission binds whenever requests queue
    budget = resident + (512 << 20)

    def run(mode, arrivals, solo=0, max_keys=1 << 26):
        dt.reset()
        tim, st = serve.wc_serve_run(ex if mode == 0 else None, dt.requests(arrivals), mode, budget,
                                     max_batch_keys=max_keys, max_batch_items=1024, max_inflight=2,
                                     solo_min_keys=solo)
        lat = (tim["completed_ns"] - arrivals).astype(np.float64) / 1e3
        return {"throughput_gkeys": keys_total / st["wall_ns"], "p50_us": float(np.percentile(lat, 50)),
                "p99_us": float(np.percentile(lat, 99)), "launches": st["launches"], "wall_ms": st["wall_ns"] / 1e6,
                "peak_admitted_bytes": st["peak_admitted_bytes"]}
    zero = np.zeros(nreq, dtype=np.uint64)
    for _ in range(max(1, args.warmup)):
        run(1, zero)
        run(0, zero)
    # batched mode: requests of 2^20 keys or more go as their own bulk calls (the per-call
    # path splits large inserts by table region) and so does a lone request; the rest queue
    # up while earlier work runs and are packed into executor batches.  The "all_in_executor"
    # runs pack every request (no solo calls), for comparison.
    solo = 1 << 20
    runs = {}
    with ClockSampler(dev.index) as clk:
        runs["per_call_closed"] = run(1, zero)
        runs["batched_closed"] = run(0, zero, solo=solo)
        runs["batched_all_in_executor_closed"] = run(0, zero)
        runs["batched_small_batches_closed"] = run(0, zero, solo=solo, max_keys=1 << 22)
        sat = nreq / (runs["per_call_closed"]["wall_ms"] * 1e-3)
        for f in (0.5, 0.8, 0.95):
            arr = wc_inputs.poisson_arrivals(0x57C00005 + int(f * 100), nreq, f * sat)
            runs["per_call_%.2f" % f] = run(1, arr)
            runs["batched_%.2f" % f] = run(0, arr, solo=solo)
            runs["batched_all_in_executor_%.2f" % f] = run(0, arr)
    b, p = runs["batched_closed"], runs["per_call_closed"]
    _common(args, "served_64tables_%dreq" % nreq, "G keys/s served (batched, closed loop)", b["throughput_gkeys"],
            "G keys/s", b["wall_ms"], "u32", {"tables": 64, "requests": nreq, "keys": keys_total,
                                              "per_call_saturation_req_per_s": sat, "hbm_budget_bytes": budget,
                                              "executor_groups": groups, "solo_min_keys": solo,
                                              "resident_table_bytes": resident}, clk,
            b["launches"], {"runs": runs, "batched_over_per_call": b["throughput_gkeys"] / p["throughput_gkeys"]})
    serve.wc_executor_destroy(ex)
    dt.close()


def run_workload(args, local_rank):
    import torch
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    {"sv32_small": run_sv32_small, "sv64_zipf": run_sv64_zipf, "mv_zipf": run_mv_zipf,
     "mv_oa_uniform_r": run_mv_oa_uniform_r, "device_api": run_device_api, "membership": run_membership,
     "served": run_served}[args.workload](args, dev)



def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload != "sv32":
        if rank == 0:
            run_workload(args, local_rank)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    run_wc(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
