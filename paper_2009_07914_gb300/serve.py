"""Binding of include/wc_exec.h (batched executor) and include/wc_serve.h (serving loop).

Argument marshalling only; the executor's persistent kernel and the serving loop are
native code in libwc.so."""
from __future__ import annotations

import ctypes

import numpy as np

from . import _binding as B


class WcWork(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("reserved", ctypes.c_int32), ("table", ctypes.c_void_p),
                ("d_keys", ctypes.c_void_p), ("d_values", ctypes.c_void_p), ("d_values_out", ctypes.c_void_p),
                ("d_found_out", ctypes.c_void_p), ("n", ctypes.c_uint64)]


class WcExecutorConfig(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("window_width", ctypes.c_int32), ("max_items", ctypes.c_uint32),
                ("tile_keys", ctypes.c_uint32), ("timeout_ns", ctypes.c_uint64), ("test_stall", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("group_insert", ctypes.c_int32), ("group_retrieve", ctypes.c_int32)]


class WcRequest(ctypes.Structure):
    _fields_ = [("work", WcWork), ("arrival_ns", ctypes.c_uint64), ("io_bytes", ctypes.c_uint64)]


class WcServeConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_uint64), ("max_batch_keys", ctypes.c_uint64),
                ("max_batch_items", ctypes.c_uint32), ("max_inflight", ctypes.c_uint32), ("mode", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("solo_min_keys", ctypes.c_uint64)]


class WcRequestTiming(ctypes.Structure):
    _fields_ = [("admitted_ns", ctypes.c_uint64), ("launched_ns", ctypes.c_uint64), ("completed_ns", ctypes.c_uint64),
                ("batch", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class WcServeStats(ctypes.Structure):
    _fields_ = [("wall_ns", ctypes.c_uint64), ("launches", ctypes.c_uint64), ("keys", ctypes.c_uint64),
                ("peak_admitted_bytes", ctypes.c_uint64), ("resident_bytes", ctypes.c_uint64)]


WC_SERVE_BATCHED = 0
WC_SERVE_PER_CALL = 1

_vp, _u32, _u64, _i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32
B.extra_signatures({
    "wc_executor_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(WcExecutorConfig)]),
    "wc_executor_destroy": (ctypes.c_int, [_vp]),
    "wc_executor_submit": (ctypes.c_int, [_vp, ctypes.POINTER(WcWork), _u32, _vp, ctypes.POINTER(_u64)]),
    "wc_executor_query": (ctypes.c_int, [_vp, _u64, ctypes.POINTER(_i32)]),
    "wc_executor_wait": (ctypes.c_int, [_vp, _u64]),
    "wc_executor_query_item": (ctypes.c_int, [_vp, _u64, _u32, ctypes.POINTER(_i32)]),
    "wc_executor_get_status": (ctypes.c_int, [_vp, ctypes.POINTER(_u32), _i32]),
    "wc_serve_run": (ctypes.c_int, [_vp, ctypes.POINTER(WcRequest), _u32, ctypes.POINTER(WcServeConfig), _vp,
                                    ctypes.POINTER(WcRequestTiming), ctypes.POINTER(WcServeStats)]),
})


def work(op: int, table: int, keys, values=None, values_out=None, found_out=None, n: int | None = None) -> WcWork:
    if n is None:
        n = keys.numel()
    return WcWork(op=op, reserved=0, table=table, d_keys=B.ptr(keys), d_values=B.ptr(values),
                  d_values_out=B.ptr(values_out), d_found_out=B.ptr(found_out), n=int(n))


def wc_executor_create(device: int, window_width: int, max_items: int = 1024, tile_keys: int = 4096,
                       timeout_ns: int = 0, test_stall: bool = False, group_insert: int = 0,
                       group_retrieve: int = 0) -> int:
    """group_insert / group_retrieve: lanes per key (0 = the defaults), e.g. the choice of
    tune.executor_groups for the served tables."""
    cfg = WcExecutorConfig(device=device, window_width=window_width, max_items=max_items, tile_keys=tile_keys,
                           timeout_ns=timeout_ns, test_stall=1 if test_stall else 0, reserved=0,
                           group_insert=group_insert, group_retrieve=group_retrieve)
    h = ctypes.c_void_p()
    B.check(B.lib().wc_executor_create(ctypes.byref(h), ctypes.byref(cfg)), "wc_executor_create")
    return int(h.value)


def wc_executor_destroy(ex: int):
    B.check(B.lib().wc_executor_destroy(ex), "wc_executor_destroy")


def wc_executor_submit(ex: int, items: list[WcWork], stream=None) -> int:
    arr = (WcWork * max(1, len(items)))(*items)
    t = ctypes.c_uint64()
    B.check(B.lib().wc_executor_submit(ex, arr, len(items), B.stream_handle(stream), ctypes.byref(t)),
            "wc_executor_submit")
    return int(t.value)


def wc_executor_query(ex: int, ticket: int) -> bool:
    d = ctypes.c_int32()
    B.check(B.lib().wc_executor_query(ex, ticket, ctypes.byref(d)), "wc_executor_query")
    return bool(d.value)


def wc_executor_query_item(ex: int, ticket: int, index: int) -> bool:
    d = ctypes.c_int32()
    B.check(B.lib().wc_executor_query_item(ex, ticket, index, ctypes.byref(d)), "wc_executor_query_item")
    return bool(d.value)


def wc_executor_wait(ex: int, ticket: int):
    B.check(B.lib().wc_executor_wait(ex, ticket), "wc_executor_wait")


def wc_executor_get_status(ex: int, clear: bool = False) -> int:
    v = ctypes.c_uint32()
    B.check(B.lib().wc_executor_get_status(ex, ctypes.byref(v), 1 if clear else 0), "wc_executor_get_status")
    return int(v.value)


def wc_serve_run(ex: int | None, requests: list[WcRequest], mode: int, hbm_budget_bytes: int,
                 max_batch_keys: int = 1 << 26, max_batch_items: int = 256, max_inflight: int = 2, stream=None,
                 solo_min_keys: int = 0):
    """Returns (timings as a dict of numpy arrays, stats dict)."""
    n = len(requests)
    arr = (WcRequest * max(1, n))(*requests)
    cfg = WcServeConfig(hbm_budget_bytes=hbm_budget_bytes, max_batch_keys=max_batch_keys,
                        max_batch_items=max_batch_items, max_inflight=max_inflight, mode=mode, reserved=0,
                        solo_min_keys=solo_min_keys)
    tim = (WcRequestTiming * max(1, n))()
    st = WcServeStats()
    B.check(B.lib().wc_serve_run(ex, arr, n, ctypes.byref(cfg), B.stream_handle(stream), tim, ctypes.byref(st)),
            "wc_serve_run")
    out = {f: np.array([getattr(tim[i], f) for i in range(n)], dtype=np.uint64)
           for f in ("admitted_ns", "launched_ns", "completed_ns", "batch")}
    return out, {f: int(getattr(st, f)) for f, _ in WcServeStats._fields_}


class DeviceTrace:
    """A serving workload materialised on the device: tables (created and pre-filled),
    and per request its key / value / output buffers.  `reset()` restores every table to
    its pre-filled content, so several modes can be run from the same start."""

    def __init__(self, trace: dict, device: int = 0, window_width: int = 8, seed: int = 0x5E7):
        import torch
        from . import api
        from .table import to_device
        self.torch, self.api = torch, api
        self.dev = torch.device("cuda", device)
        self.trace = trace
        self.tables = [api.wc_table_create(0, 4, 4, int(c), window_width, 0, seed + i, device)
                       for i, c in enumerate(trace["caps"])]
        self.pf = [(to_device(k, 4, self.dev), to_device(v, 4, self.dev))
                   for k, v in zip(trace["prefill_keys"], trace["prefill_vals"])]
        self.bufs = []
        for r in trace["requests"]:
            k = to_device(r["keys"], 4, self.dev)
            v = to_device(r["values"], 4, self.dev) if r["op"] == 0 else None
            o = torch.empty(k.numel(), dtype=torch.int32, device=self.dev) if r["op"] == 1 else None
            f = torch.empty(k.numel(), dtype=torch.uint8, device=self.dev) if r["op"] == 1 else None
            self.bufs.append((k, v, o, f))

    def reset(self):
        s = self.torch.cuda.current_stream()
        for h, (k, v) in zip(self.tables, self.pf):
            self.api.wc_table_clear(h, s)
            if k.numel():
                self.api.wc_insert(h, k, v, stream=s)
        for (_, _, o, f) in self.bufs:
            if o is not None:
                o.fill_(0)
                f.fill_(2)
        self.torch.cuda.synchronize()

    def works(self):
        out = []
        for r, (k, v, o, f) in zip(self.trace["requests"], self.bufs):
            out.append(work(r["op"], self.tables[r["table"]], k, v, o, f))
        return out

    def requests(self, arrivals_ns):
        out = []
        for w, (k, v, o, f), a in zip(self.works(), self.bufs, arrivals_ns):
            io = sum(x.numel() * x.element_size() for x in (k, v, o, f) if x is not None)
            out.append(WcRequest(work=w, arrival_ns=int(a), io_bytes=io))
        return out

    def retrieve_results(self):
        return [(o.cpu().numpy().view(np.uint32), f.cpu().numpy()) if o is not None else None
                for (_, _, o, f) in self.bufs]

    def sizes(self):
        return [self.api.wc_size(h) for h in self.tables]

    def close(self):
        self.torch.cuda.synchronize()
        for h in self.tables:
            self.api.wc_table_destroy(h)
        self.tables = []
