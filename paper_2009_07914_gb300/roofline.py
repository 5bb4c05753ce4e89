"""Binding of include/wc_roofline.h: random-access probes that measure the bound of the
hash-table hot path (random window reads; read + CAS for inserts) on this device."""
from __future__ import annotations

import ctypes

import torch

from . import _binding as B


class WcRandAccessConfig(ctypes.Structure):
    _fields_ = [("buffer_bytes", ctypes.c_uint64), ("accesses", ctypes.c_uint64), ("seed", ctypes.c_uint64),
                ("access_bytes", ctypes.c_uint32), ("mode", ctypes.c_uint32), ("block_threads", ctypes.c_uint32),
                ("blocks_per_sm", ctypes.c_uint32), ("in_flight", ctypes.c_uint32), ("lanes", ctypes.c_uint32)]


B.extra_signatures({
    "wc_bench_random_access": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(WcRandAccessConfig), ctypes.c_void_p,
                                              ctypes.c_void_p]),
    "wc_set_l2_fetch_granularity": (ctypes.c_int, [ctypes.c_int32]),
    "wc_get_l2_fetch_granularity": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int32)]),
    "wc_bench_device_api": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint32,
                                           ctypes.c_void_p, ctypes.c_void_p]),
    "wc_bench_mv_append": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                          ctypes.c_void_p]),
    "wc_bench_device_api_group": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
                                                 ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p]),
})


def wc_bench_device_api_group(table: int, mode: int, group: int, n: int, key_seed: int,
                              sink: torch.Tensor | None = None, stream=None):
    """Device-API probe with tiles of `group` threads per key: mode 0 insert, 1 lookup."""
    B.check(B.lib().wc_bench_device_api_group(table, mode, group, n, key_seed & 0xFFFFFFFF,
                                              None if sink is None else B.ptr(sink), B.stream_handle(stream)),
            "wc_bench_device_api_group")


def wc_bench_mv_append(table: int, keys: torch.Tensor, values: torch.Tensor, n: int | None = None, stream=None):
    """Device-API probe: one thread per pair appends to a bucket multi-value table."""
    n = keys.numel() if n is None else n
    B.check(B.lib().wc_bench_mv_append(table, B.ptr(keys), B.ptr(values), n, B.stream_handle(stream)),
            "wc_bench_mv_append")


def wc_bench_random_access(buffer: torch.Tensor, access_bytes: int, mode: int, accesses: int, sink: torch.Tensor,
                           seed: int = 1, buffer_bytes: int | None = None, block_threads: int = 0,
                           blocks_per_sm: int = 0, in_flight: int = 0, lanes: int = 0, stream=None):
    nbytes = buffer.numel() * buffer.element_size() if buffer_bytes is None else buffer_bytes
    nbytes -= nbytes % access_bytes
    cfg = WcRandAccessConfig(buffer_bytes=nbytes, accesses=accesses, seed=seed, access_bytes=access_bytes, mode=mode,
                             block_threads=block_threads, blocks_per_sm=blocks_per_sm, in_flight=in_flight,
                             lanes=lanes)
    B.check(B.lib().wc_bench_random_access(B.ptr(buffer), ctypes.byref(cfg), B.ptr(sink), B.stream_handle(stream)),
            "wc_bench_random_access")


def wc_set_l2_fetch_granularity(nbytes: int):
    B.check(B.lib().wc_set_l2_fetch_granularity(int(nbytes)), "wc_set_l2_fetch_granularity")


def wc_get_l2_fetch_granularity() -> int:
    v = ctypes.c_int32()
    B.check(B.lib().wc_get_l2_fetch_granularity(ctypes.byref(v)), "wc_get_l2_fetch_granularity")
    return int(v.value)


def wc_bench_device_api(table: int, mode: int, n: int, key_seed: int, sink: torch.Tensor | None = None,
                        stream=None):
    """Device-API probe (include/wc_roofline.h): mode 0 fused insert, mode 1 fused lookup."""
    B.check(B.lib().wc_bench_device_api(table, mode, n, key_seed & 0xFFFFFFFF, None if sink is None else B.ptr(sink),
                                        B.stream_handle(stream)), "wc_bench_device_api")


def random_access_rate(buffer: torch.Tensor, access_bytes: int, mode: int = 0, accesses: int = 1 << 28,
                       reps: int = 3, buffer_bytes: int | None = None, **kw) -> dict:
    """Best-of-`reps` rate of random `access_bytes` reads (mode 1: read + CAS) over
    `buffer`, timed with CUDA events on the current stream (one warm-up launch)."""
    sink = torch.zeros(1, dtype=torch.int64, device=buffer.device)
    s = torch.cuda.current_stream()
    wc_bench_random_access(buffer, access_bytes, mode, accesses, sink, seed=99, buffer_bytes=buffer_bytes, **kw)
    best = None
    for r in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        wc_bench_random_access(buffer, access_bytes, mode, accesses, sink, seed=100 + r, buffer_bytes=buffer_bytes,
                               **kw)
        b.record(s)
        b.synchronize()
        ms = a.elapsed_time(b)
        best = ms if best is None else min(best, ms)
    return {"access_bytes": access_bytes, "mode": mode, "ms": best, "accesses_per_s": accesses / (best * 1e-3),
            "gbs": accesses * access_bytes / (best * 1e-3) / 1e9}


def best_rate(buffer: torch.Tensor, access_bytes: int, mode: int, accesses: int, buffer_bytes: int | None = None,
              in_flight=(4, 8, 16), lanes=(1, 2), reps: int = 2) -> dict:
    """The highest rate of random `access_bytes` accesses (mode 0 read, 1 read + CAS) over
    every shape of in_flight x lanes: the memory system's ceiling for this access, not
    the limit of one probe shape."""
    best = None
    for u in in_flight:
        for g in lanes:
            if access_bytes // g < 8:
                continue
            r = random_access_rate(buffer, access_bytes, mode, accesses, reps=reps, buffer_bytes=buffer_bytes,
                                   in_flight=u, lanes=g)
            r.update(in_flight=u, lanes=g)
            if best is None or r["accesses_per_s"] > best["accesses_per_s"]:
                best = r
    return best


def main():
    """Sweep of the random-access roofline: rate vs access size, mode, buffer size and L2
    fetch-granularity limit (one JSON line per point)."""
    import argparse
    import json
    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--accesses", type=int, default=1 << 27)
    ap.add_argument("--gran", default="32,64,128", help="L2 fetch-granularity limits to try")
    ap.add_argument("--bytes", default="32,64,128")
    ap.add_argument("--buffers-mib", default="8192,1024,64")
    ap.add_argument("--capacity-curve", action="store_true",
                    help="also sweep 64 B reads / read+CAS over buffers of 4 MiB .. 1 GiB")
    ap.add_argument("--mlp-sweep", action="store_true",
                    help="only: rate vs accesses in flight per thread (1..16) and lanes per access (1, 2, 4) for "
                         "--bytes reads and read+CAS over --buffers-mib, at the default fetch granularity")
    ap.add_argument("--in-flight", default="1,2,4,8,16", help="--mlp-sweep: accesses in flight per thread")
    ap.add_argument("--lanes", default="1,2,4", help="--mlp-sweep: lanes per access")
    ap.add_argument("--modes", default="0,1", help="--mlp-sweep: 0 read, 1 read + CAS")
    a = ap.parse_args()
    bufs = [int(x) for x in a.buffers_mib.split(",")]
    dev = torch.device("cuda", torch.cuda.current_device())
    buf = torch.zeros(max(bufs + [1024]) << 20, dtype=torch.uint8, device=dev)
    if a.mlp_sweep:
        for ab in (int(x) for x in a.bytes.split(",")):
            for mode in (int(x) for x in a.modes.split(",")):
                for mib in bufs:
                    for u in (int(x) for x in a.in_flight.split(",")):
                        for g in (int(x) for x in a.lanes.split(",")):
                            if ab // g < 8:
                                continue
                            r = random_access_rate(buf, ab, mode, a.accesses, reps=2, buffer_bytes=mib << 20,
                                                   in_flight=u, lanes=g)
                            r.update(buffer_mib=mib, in_flight=u, lanes=g)
                            print(json.dumps(r), flush=True)
        return
    for g in (int(x) for x in a.gran.split(",")):
        wc_set_l2_fetch_granularity(g)
        for ab in (int(x) for x in a.bytes.split(",")):
            for mode in (0, 1):
                for mib in bufs:
                    r = random_access_rate(buf, ab, mode, a.accesses, buffer_bytes=mib << 20)
                    r.update(gran=g, buffer_mib=mib)
                    print(json.dumps(r), flush=True)
    if a.capacity_curve:
        for mode in (0, 1):
            for mib in (4, 8, 16, 24, 32, 48, 64, 80, 96, 128, 192, 256, 512, 1024):
                r = random_access_rate(buf, 64, mode, a.accesses // 2, buffer_bytes=mib << 20)
                r.update(curve=True, buffer_mib=mib)
                print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
