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
    ap.add_argument("--group", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def source_digest():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2009_07914_gb300", "csrc")
    for name in sorted(os.listdir(d)):
        with open(os.path.join(d, name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, workload: str):
    """dram bytes per launch of `kernel` from the committed ncu summary, if it was taken
    on the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            rows = json.load(f)
    except Exception:
        return None
    for r in rows:
        if r.get("kernel") == kernel and r.get("workload") == workload and r.get("source") == source_digest():
            return r.get("dram_bytes_per_launch")
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


def cpu_baseline(log2n_sample: int, alpha: float):
    """The oracle (single-threaded std::unordered_map, reserve(n)) on a bounded sample of
    the same workload: insert n pairs then retrieve n queries (half absent)."""
    import oracle
    n = 1 << log2n_sample
    d = wc_inputs.sv_insert_retrieve_u32(SEED, n, n // 2, n // 2)
    o = oracle.SingleValue(4, 4)
    o.reserve(int(n / alpha))
    t0 = time.perf_counter()
    o.insert(d["keys"], d["values"])
    t1 = time.perf_counter()
    o.retrieve(d["queries"])
    t2 = time.perf_counter()
    return {"value": 2 * n / (t2 - t0) / 1e9, "unit": "G ops/s", "cores": 1, "kind": "oracle",
            "sample": "2^%d inserts + 2^%d retrievals (half absent), std::unordered_map, one host thread"
                      % (log2n_sample, log2n_sample),
            "insert_gops": n / (t1 - t0) / 1e9, "retrieve_gops": n / (t2 - t1) / 1e9}


def run_reference(args, rank, world):
    if rank != 0:
        return
    steps, warm = args.steps, args.warmup
    log2s = 21
    vals = []
    for i in range(warm + steps):
        r = cpu_baseline(log2s, args.alpha)
        if i >= warm:
            vals.append(r)
    v = statistics.mean(x["value"] for x in vals)
    sample = vals[0]["sample"]
    ms = 2 * (1 << log2s) / (v * 1e9) * 1e3
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "G ops/s", "n_gpus": args.gpus,
        "steps": steps, "warmup": warm, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "sv_u32_n2^%d_alpha%.2f" % (args.log2n, args.alpha), "sample_log2n": log2s},
        "cpu_baseline": {"value": v, "unit": "G ops/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "G ops/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "insert_gops": statistics.mean(x["insert_gops"] for x in vals),
        "retrieve_gops": statistics.mean(x["retrieve_gops"] for x in vals),
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
    h = api.wc_table_create(wc.WC_SINGLE_VALUE, 4, 4, int(np.ceil(n / args.alpha)), args.window, 0,
                            0x5EEDC0DE + rank, local_rank)
    info = api.wc_table_get_info(h)
    if args.group:
        for op in (wc.WC_OP_INSERT, wc.WC_OP_RETRIEVE, wc.WC_OP_ERASE):
            api.wc_table_set_launch(h, op, args.group)
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
    if world > 1:
        tt = torch.tensor([total_ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = float(tt.item())
    ms_step = total_ms / args.steps
    value = world * 2 * n / (ms_step * 1e-3) / 1e9

    # end-to-end through the C ABI from pinned host buffers (H2D, insert, retrieve, D2H)
    e2e = None
    if not args.no_e2e:
        hk = torch.from_numpy(d["keys"].view(np.int32)).pin_memory()
        hv = torch.from_numpy(d["values"].view(np.int32)).pin_memory()
        hq = torch.from_numpy(d["queries"].view(np.int32)).pin_memory()
        ho = torch.empty(n, dtype=torch.int32).pin_memory()
        hf = torch.empty(n, dtype=torch.uint8).pin_memory()
        dk, dv, dq = torch.empty_like(keys), torch.empty_like(vals), torch.empty_like(qk)

        def e2e_step():
            api.wc_table_clear(h, s)
            dk.copy_(hk, non_blocking=True)
            dv.copy_(hv, non_blocking=True)
            api.wc_insert(h, dk, dv, n, s)
            dq.copy_(hq, non_blocking=True)
            api.wc_retrieve(h, dq, out, found, n, s)
            ho.copy_(out, non_blocking=True)
            hf.copy_(found, non_blocking=True)
        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        assert np.array_equal(hf.numpy(), found.cpu().numpy())
        k = max(1, args.steps // 2)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        for _ in range(k):
            e2e_step()
        b.record(s)
        torch.cuda.synchronize()
        e_ms = a.elapsed_time(b) / k
        e2e = {"value": world * 2 * n / (e_ms * 1e-3) / 1e9, "unit": "G ops/s",
               "h2d_bytes_per_step": n * 4 * 3, "d2h_bytes_per_step": n * 5, "ms_per_step": e_ms}

    if rank != 0:
        return
    peak, peak_kind = peaks()
    ins, ret = statistics.median(ins_ms), statistics.median(ret_ms)
    dom = "insert" if ins >= ret else "retrieve"
    dom_ms = max(ins, ret)
    achieved = BYTES_PER_OP[dom] * n / (dom_ms * 1e-3) / 1e9
    workload_name = "sv_u32_n2^%d_alpha%.2f" % (args.log2n, args.alpha)
    kname = "k_sv_insert" if dom == "insert" else "k_sv_retrieve"
    traffic = ncu_traffic(kname, workload_name)
    cpu = None if args.no_cpu else cpu_baseline(23, args.alpha)
    res = {
        "metric": METRIC, "value": value, "unit": "G ops/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": workload_name, "n": n, "queries": n, "present_fraction": 0.5,
                   "capacity": info["capacity"], "achieved_alpha": n / info["capacity"],
                   "window_slots": info["window_width"], "group_insert": g_ins, "group_retrieve": g_ret,
                   "table_bytes": info["table_bytes"],
                   "l2": "no flush: inputs and table larger than L2 (table %.2f GB, keys %.2f GB)"
                         % (info["table_bytes"] / 1e9, n * 4 / 1e9),
                   "parallelism": "replicas (independent table per GPU)"},
        "insert_gops": n / (ins * 1e-3) / 1e9, "retrieve_gops": n / (ret * 1e-3) / 1e9,
        "clear_ms": statistics.median(clear_ms), "insert_ms": ins, "retrieve_ms": ret,
        "roofline": {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_kind": peak_kind,
                     "bytes_per_op": BYTES_PER_OP[dom], "traffic": traffic},
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": 2 * args.steps, "clocks": clk.summary(),
    }
    print(json.dumps(res), flush=True)
    api.wc_table_destroy(h)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
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
