"""Python functions with the names of the C ABI (include/wc.h).

Each function marshals its arguments (tensor -> device address, stream -> handle,
ctypes out-parameters) and calls the library once.  Tables are opaque integer handles.
Buffers are torch tensors of any 4- or 8-byte integer dtype: the library reads their
bytes, so uint32 keys may travel as int32 tensors.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _binding as B
from ._binding import (WC_BLOOM_FILTER, WC_COUNTING, WC_HASH_SET, WC_MULTI_VALUE, WC_MULTI_VALUE_OA,
                       WC_OPT_OVERFLOW_BITS, WC_OPT_SOA, WC_SINGLE_VALUE, WcLaunch,
                       WcTableConfig, WcTableInfo, check, lib, ptr, stream_handle)

__all__ = [
    "wc_plan_capacity", "wc_table_create", "wc_table_destroy", "wc_table_clear", "wc_table_get_info",
    "wc_table_set_launch", "wc_table_get_launch", "wc_insert", "wc_retrieve", "wc_erase", "wc_count_values",
    "wc_retrieve_multi", "wc_size", "wc_num_keys", "wc_load_factor", "wc_get_status", "wc_status_string",
    "wc_insert_noalloc", "WC_NOALLOC_SCRATCH_BYTES", "wc_value_pool_used", "wc_contains", "wc_insert_host",
    "wc_retrieve_host",
]


def _n_of(n, t: torch.Tensor | None, width: int | None = None) -> int:
    if n is None:
        if not isinstance(t, torch.Tensor):
            raise ValueError("n is required when the keys are a raw address")
        n = t.numel()
    if isinstance(t, torch.Tensor):
        if t.numel() < n:
            raise ValueError("buffer holds %d elements, n = %d" % (t.numel(), n))
        if width is not None and t.numel() and t.element_size() != width:
            raise ValueError("element width %d, table expects %d" % (t.element_size(), width))
        if t.numel() and not t.is_cuda:
            raise ValueError("device buffers must be CUDA tensors")
    return int(n)


def wc_status_string(code: int) -> str:
    return B.status_string(code)


def wc_plan_capacity(min_capacity: int, window_width: int) -> tuple[int, int]:
    p, c = ctypes.c_uint64(), ctypes.c_uint64()
    check(lib().wc_plan_capacity(int(min_capacity), int(window_width), ctypes.byref(p), ctypes.byref(c)),
          "wc_plan_capacity")
    return int(p.value), int(c.value)


def wc_table_create(kind: int = WC_SINGLE_VALUE, key_bytes: int = 4, value_bytes: int = 4, min_capacity: int = 1024,
                    window_width: int = 0, value_pool_capacity: int = 0, seed: int = 0x5EED_C0DE,
                    device: int | None = None, l2_persist: bool = False, options: int = 0,
                    bucket_first_size: int = 0, bucket_growth: float = 1.0) -> int:
    if device is None:
        device = torch.cuda.current_device()
    cfg = WcTableConfig(kind=kind, key_bytes=key_bytes, value_bytes=value_bytes, window_width=window_width,
                        device=device, l2_persist=1 if l2_persist else 0, options=int(options), reserved=0,
                        min_capacity=int(min_capacity),
                        value_pool_capacity=int(value_pool_capacity), seed=int(seed) & (2 ** 64 - 1),
                        bucket_first_size=int(bucket_first_size), bucket_growth=float(bucket_growth))
    h = ctypes.c_void_p()
    check(lib().wc_table_create(ctypes.byref(h), ctypes.byref(cfg)), "wc_table_create")
    return int(h.value)


def wc_table_destroy(t: int):
    check(lib().wc_table_destroy(t), "wc_table_destroy")


def wc_table_clear(t: int, stream=None):
    check(lib().wc_table_clear(t, stream_handle(stream)), "wc_table_clear")


def wc_table_get_info(t: int) -> dict:
    info = WcTableInfo()
    check(lib().wc_table_get_info(t, ctypes.byref(info)), "wc_table_get_info")
    return {f: getattr(info, f) for f, _ in WcTableInfo._fields_}


def wc_table_set_launch(t: int, op: int, group_size: int, block_threads: int = 256, blocks_per_sm: int = 0,
                        scheme: int = 0, region_mib: int = 0, keys_in_flight: int = 0):
    lc = WcLaunch(group_size=group_size, block_threads=block_threads, blocks_per_sm=blocks_per_sm, scheme=scheme,
                  region_mib=region_mib, keys_in_flight=keys_in_flight)
    check(lib().wc_table_set_launch(t, op, ctypes.byref(lc)), "wc_table_set_launch")


def wc_table_get_launch(t: int, op: int) -> dict:
    lc = WcLaunch()
    check(lib().wc_table_get_launch(t, op, ctypes.byref(lc)), "wc_table_get_launch")
    return {f: getattr(lc, f) for f, _ in WcLaunch._fields_}


class WcTuning(ctypes.Structure):
    """include/wc_tune.h wc_tuning."""
    _fields_ = [("window_width", ctypes.c_int32), ("candidates", ctypes.c_int32), ("from_cache", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("launch", WcLaunch * 3), ("ms", ctypes.c_double * 3),
                ("sample_keys", ctypes.c_uint64), ("load", ctypes.c_double)]


B.extra_signatures({
    "wc_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_uint64, ctypes.c_int32,
                                   ctypes.c_void_p]),
    "wc_table_apply_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "wc_autotune_sample_keys": (ctypes.c_uint64, [ctypes.c_void_p]),
})


def _tuning_dict(tu: WcTuning) -> dict:
    return {"window_width": tu.window_width, "candidates": tu.candidates, "from_cache": tu.from_cache,
            "launch": [{f: getattr(tu.launch[i], f) for f, _ in WcLaunch._fields_} for i in range(3)],
            "ms": [tu.ms[i] for i in range(3)], "sample_keys": tu.sample_keys, "load": tu.load}


def wc_autotune(kind: int = WC_SINGLE_VALUE, key_bytes: int = 4, value_bytes: int = 4, window_width: int = 0,
                load: float = 0.9, sample_keys: int = 1 << 20, options: int = 0, use_cache: bool = True,
                device: int | None = None, seed: int = 0x5EED_C0DE) -> dict:
    """Time the library's kernels on a synthetic sample and return the chosen window width
    and launch shapes (wc_tune.h); launch[i] is for op i (insert, retrieve, erase)."""
    if device is None:
        device = torch.cuda.current_device()
    cfg = WcTableConfig(kind=kind, key_bytes=key_bytes, value_bytes=value_bytes, window_width=window_width,
                        device=device, l2_persist=0, options=int(options), reserved=0, min_capacity=0,
                        value_pool_capacity=0, seed=int(seed) & (2 ** 64 - 1), bucket_first_size=0,
                        bucket_growth=1.0)
    tu = WcTuning()
    check(lib().wc_autotune(ctypes.byref(cfg), float(load), int(sample_keys), 1 if use_cache else 0,
                            ctypes.byref(tu)), "wc_autotune")
    return _tuning_dict(tu)


def wc_autotune_sample_keys(kind: int = WC_SINGLE_VALUE, key_bytes: int = 4, value_bytes: int = 4,
                            min_capacity: int = 1024, options: int = 0) -> int:
    """Sample size wc_table_create tunes on for window_width = 0 (at load 0.9)."""
    cfg = WcTableConfig(kind=kind, key_bytes=key_bytes, value_bytes=value_bytes, window_width=0, device=0,
                        l2_persist=0, options=int(options), reserved=0, min_capacity=int(min_capacity),
                        value_pool_capacity=0, seed=0, bucket_first_size=0, bucket_growth=1.0)
    return int(lib().wc_autotune_sample_keys(ctypes.byref(cfg)))


def wc_table_apply_tuning(t: int, tuning: dict):
    tu = WcTuning(window_width=tuning["window_width"], candidates=tuning.get("candidates", 0),
                  from_cache=tuning.get("from_cache", 0), reserved=0, sample_keys=tuning.get("sample_keys", 0),
                  load=tuning.get("load", 0.0))
    for i in range(3):
        for f, _ in WcLaunch._fields_:
            setattr(tu.launch[i], f, int(tuning["launch"][i][f]))
        tu.ms[i] = float(tuning.get("ms", [0, 0, 0])[i])
    check(lib().wc_table_apply_tuning(t, ctypes.byref(tu)), "wc_table_apply_tuning")


def wc_insert(t: int, keys, values, n: int | None = None, stream=None):
    """values may be None for counting tables (every key counts 1)."""
    n = _n_of(n, keys)
    if values is not None:
        _n_of(n, values)
    check(lib().wc_insert(t, ptr(keys), ptr(values), n, stream_handle(stream)), "wc_insert")


B.extra_signatures({"wc_insert_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                          ctypes.c_uint64, ctypes.c_void_p])})

WC_NOALLOC_SCRATCH_BYTES = 16 << 20


def wc_insert_noalloc(t: int, keys, values, n: int | None = None, stream=None):
    """wc_insert for callers that cannot allocate: splits the batch in the library's
    fixed device buffer (at most WC_NOALLOC_SCRATCH_BYTES / (key + value bytes) pairs,
    minus a few); calls on one device must not overlap on the GPU."""
    n = _n_of(n, keys)
    _n_of(n, values)
    check(lib().wc_insert_noalloc(t, ptr(keys), ptr(values), n, stream_handle(stream)), "wc_insert_noalloc")


def wc_retrieve(t: int, keys, values_out, found_out=None, n: int | None = None, stream=None):
    n = _n_of(n, keys)
    _n_of(n, values_out)
    if found_out is not None:
        _n_of(n, found_out, 1)
    check(lib().wc_retrieve(t, ptr(keys), n, ptr(values_out), ptr(found_out), stream_handle(stream)),
          "wc_retrieve")


def _host_ptr(x) -> int | None:
    """Address of a host buffer: a CPU tensor (pinned for full speed) or a numpy array."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, torch.Tensor):
        if x.is_cuda:
            raise ValueError("host buffers must be CPU tensors")
        if x.numel() and not x.is_contiguous():
            raise ValueError("buffers must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("buffers must be contiguous")
        return x.ctypes.data
    raise TypeError("expected a CPU tensor, a numpy array or an integer address, got %r" % type(x))


def wc_insert_host(t: int, keys, values, n: int | None = None, stream=None):
    """wc_insert from host buffers (pinned CPU tensors or numpy arrays)."""
    n = len(keys) if n is None else int(n)
    check(lib().wc_insert_host(t, _host_ptr(keys), _host_ptr(values), n, stream_handle(stream)), "wc_insert_host")


def wc_retrieve_host(t: int, keys, values_out, found_out=None, n: int | None = None, stream=None):
    """wc_retrieve from and into host buffers; the results are there once `stream` is."""
    n = len(keys) if n is None else int(n)
    check(lib().wc_retrieve_host(t, _host_ptr(keys), n, _host_ptr(values_out), _host_ptr(found_out),
                                 stream_handle(stream)), "wc_retrieve_host")


def wc_contains(t: int, keys, found_out, n: int | None = None, stream=None):
    n = _n_of(n, keys)
    _n_of(n, found_out)
    check(lib().wc_contains(t, ptr(keys), n, ptr(found_out), stream_handle(stream)), "wc_contains")


def wc_erase(t: int, keys, n: int | None = None, stream=None):
    n = _n_of(n, keys)
    check(lib().wc_erase(t, ptr(keys), n, stream_handle(stream)), "wc_erase")


def wc_count_values(t: int, keys, offsets_out, n: int | None = None, want_total: bool = True, stream=None):
    """Fills offsets_out[0..n] (n+1 uint64); returns the total if want_total (blocking)."""
    n = _n_of(n, keys)
    _n_of(n + 1, offsets_out, 8)
    total = ctypes.c_uint64()
    check(lib().wc_count_values(t, ptr(keys), n, ptr(offsets_out), ctypes.byref(total) if want_total else None,
                                stream_handle(stream)), "wc_count_values")
    return int(total.value) if want_total else None


def wc_retrieve_multi(t: int, keys, offsets, values_out, n: int | None = None, stream=None):
    n = _n_of(n, keys)
    _n_of(n + 1, offsets, 8)
    check(lib().wc_retrieve_multi(t, ptr(keys), n, ptr(offsets), ptr(values_out), stream_handle(stream)),
          "wc_retrieve_multi")


def _read_u64(fn, t, stream, where):
    v = ctypes.c_uint64()
    check(fn(t, ctypes.byref(v), stream_handle(stream)), where)
    return int(v.value)


def wc_size(t: int, stream=None) -> int:
    return _read_u64(lib().wc_size, t, stream, "wc_size")


def wc_num_keys(t: int, stream=None) -> int:
    return _read_u64(lib().wc_num_keys, t, stream, "wc_num_keys")


def wc_value_pool_used(t: int, stream=None) -> int:
    return _read_u64(lib().wc_value_pool_used, t, stream, "wc_value_pool_used")


def wc_load_factor(t: int, stream=None) -> float:
    v = ctypes.c_double()
    check(lib().wc_load_factor(t, ctypes.byref(v), stream_handle(stream)), "wc_load_factor")
    return float(v.value)


def wc_get_status(t: int, clear: bool = False, stream=None) -> int:
    v = ctypes.c_uint32()
    check(lib().wc_get_status(t, ctypes.byref(v), 1 if clear else 0, stream_handle(stream)), "wc_get_status")
    return int(v.value)


def wc_check_status(t: int, stream=None) -> tuple[int, int]:
    """(wc_status code, raw flag bits); the word is cleared.  Does not raise for the
    device conditions (WC_ERR_FULL / WC_ERR_TIMEOUT are returned as the code)."""
    v = ctypes.c_uint32()
    code = lib().wc_check_status(t, ctypes.byref(v), stream_handle(stream))
    if code not in (B.WC_OK, B.WC_ERR_FULL, B.WC_ERR_TIMEOUT):
        check(code, "wc_check_status")
    return int(code), int(v.value)


def wc_table_dump_slots(t: int, stream=None) -> np.ndarray:
    """Host copy of the slot array as bytes (slot i at byte i * slot_bytes)."""
    info = wc_table_get_info(t)
    out = np.empty(info["table_bytes"], dtype=np.uint8)
    check(lib().wc_table_dump_slots(t, out.ctypes.data, out.size, stream_handle(stream)), "wc_table_dump_slots")
    return out


def wc_table_device_view(t: int) -> B.WcDeviceView:
    """The table's wc_device_view (device pointers and geometry for user kernels)."""
    v = B.WcDeviceView()
    check(lib().wc_table_device_view(t, ctypes.byref(v)), "wc_table_device_view")
    return v


def wc_table_dump_overflow_bits(t: int, stream=None) -> np.ndarray:
    """Host copy of a table's overflow bits: uint32 words holding one byte per window
    (window w in byte w, little-endian), bit g of a byte = keys of tag g walked past."""
    info = wc_table_get_info(t)
    out = np.empty((info["windows"] + 3) // 4, dtype=np.uint32)
    check(lib().wc_table_dump_overflow_bits(t, out.ctypes.data, out.size, stream_handle(stream)),
          "wc_table_dump_overflow_bits")
    return out


def wc_table_snapshot_bytes(t: int) -> int:
    return int(lib().wc_table_snapshot_bytes(t))


def wc_table_snapshot(t: int, stream=None) -> np.ndarray:
    out = np.empty(wc_table_snapshot_bytes(t), dtype=np.uint8)
    check(lib().wc_table_snapshot(t, out.ctypes.data, out.size, stream_handle(stream)), "wc_table_snapshot")
    return out


def wc_table_restore(t: int, snapshot: np.ndarray, stream=None):
    buf = np.ascontiguousarray(snapshot).view(np.uint8)
    check(lib().wc_table_restore(t, buf.ctypes.data, buf.size, stream_handle(stream)), "wc_table_restore")


def wc_debug_fail_allocations(count: int):
    check(lib().wc_debug_fail_allocations(count), "wc_debug_fail_allocations")


__all__ += ["wc_check_status", "wc_table_dump_slots", "wc_table_device_view", "wc_table_dump_overflow_bits",
            "wc_table_snapshot_bytes",
            "wc_table_snapshot",
            "wc_table_restore", "wc_debug_fail_allocations"]
__all__ += ["WC_SINGLE_VALUE", "WC_MULTI_VALUE", "WC_MULTI_VALUE_OA", "WC_HASH_SET", "WC_COUNTING",
            "WC_BLOOM_FILTER", "WC_OPT_OVERFLOW_BITS", "WC_OPT_SOA"]
