"""ctypes binding of libwc.so (the C ABI declared in include/wc.h).

Argument marshalling only: device buffers are torch tensors (or raw integer device
pointers), streams are torch.cuda.Stream objects (None = torch's current stream).
Every computation happens in the library's CUDA kernels; there is no fallback path.
If libwc.so is missing this module raises, it never substitutes anything.
"""
from __future__ import annotations

import ctypes
import os

import torch  # loads the shared CUDA runtime the library links against

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libwc.so")

WC_OK = 0
WC_ERR_INVALID_ARG = 1
WC_ERR_OUT_OF_MEMORY = 2
WC_ERR_FULL = 3
WC_ERR_CUDA = 4
WC_ERR_TIMEOUT = 5
WC_ERR_UNSUPPORTED = 6

WC_FLAG_DUPLICATE_KEY = 1
WC_FLAG_INVALID_KEY = 2
WC_FLAG_PROBE_LIMIT = 4
WC_FLAG_POOL_EXHAUSTED = 8
WC_FLAG_COUNT_OVERFLOW = 16
WC_FLAG_QUEUE_TIMEOUT = 32

WC_SINGLE_VALUE = 0
WC_MULTI_VALUE = 1
WC_MULTI_VALUE_OA = 2
WC_HASH_SET = 3
WC_COUNTING = 4
WC_BLOOM_FILTER = 5
WC_OPT_OVERFLOW_BITS = 1
WC_OPT_SOA = 2

WC_SCHEME_AUTO = 0
WC_SCHEME_DIRECT = 1
WC_SCHEME_BLOCKED = 2
WC_SCHEME_DEDUP = 3

WC_OP_INSERT = 0
WC_OP_RETRIEVE = 1
WC_OP_ERASE = 2
WC_OP_COUNT = 3


class WcTableConfig(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("key_bytes", ctypes.c_int32), ("value_bytes", ctypes.c_int32),
                ("window_width", ctypes.c_int32), ("device", ctypes.c_int32), ("l2_persist", ctypes.c_int32),
                ("options", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("min_capacity", ctypes.c_uint64), ("value_pool_capacity", ctypes.c_uint64),
                ("seed", ctypes.c_uint64), ("bucket_first_size", ctypes.c_uint64), ("bucket_growth", ctypes.c_double)]


class WcTableInfo(ctypes.Structure):
    _fields_ = [("capacity", ctypes.c_uint64), ("windows", ctypes.c_uint64), ("slot_bytes", ctypes.c_uint64),
                ("table_bytes", ctypes.c_uint64), ("pool_capacity", ctypes.c_uint64),
                ("device_bytes", ctypes.c_uint64), ("window_width", ctypes.c_int32), ("kind", ctypes.c_int32),
                ("options", ctypes.c_int32), ("reserved", ctypes.c_int32), ("work_bytes", ctypes.c_uint64)]


class WcDeviceView(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_void_p), ("status", ctypes.c_void_p), ("size", ctypes.c_void_p),
                ("overflow_bits", ctypes.c_void_p), ("seed", ctypes.c_uint64), ("capacity", ctypes.c_uint64),
                ("windows", ctypes.c_uint32), ("window_width", ctypes.c_uint32), ("kind", ctypes.c_int32),
                ("key_bytes", ctypes.c_int32), ("value_bytes", ctypes.c_int32), ("slot_bytes", ctypes.c_int32),
                ("pool", ctypes.c_void_p), ("pool_cursor", ctypes.c_void_p), ("num_keys", ctypes.c_void_p),
                ("bucket_cum_size", ctypes.c_void_p), ("bucket_cum_foot", ctypes.c_void_p),
                ("pool_capacity", ctypes.c_uint64), ("bucket_size", ctypes.c_uint64),
                ("bucket_foot0", ctypes.c_uint64), ("bucket_foot", ctypes.c_uint64),
                ("bucket_count", ctypes.c_uint32), ("growth", ctypes.c_int32), ("wait_ns", ctypes.c_uint64)]


class WcLaunch(ctypes.Structure):
    _fields_ = [("group_size", ctypes.c_int32), ("block_threads", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("scheme", ctypes.c_int32), ("region_mib", ctypes.c_int32),
                ("keys_in_flight", ctypes.c_int32)]


class WcError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__("%s: %s (wc_status %d)" % (where, status_string(code), code))


_lib = None

# name -> (restype, argtypes); mirrors include/wc.h
_vp, _u64, _i32, _u32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int32, ctypes.c_uint32
_SIGS = {
    "wc_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "wc_plan_capacity": (ctypes.c_int, [_u64, _i32, ctypes.POINTER(_u64), ctypes.POINTER(_u64)]),
    "wc_table_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(WcTableConfig)]),
    "wc_table_destroy": (ctypes.c_int, [_vp]),
    "wc_table_clear": (ctypes.c_int, [_vp, _vp]),
    "wc_table_get_info": (ctypes.c_int, [_vp, ctypes.POINTER(WcTableInfo)]),
    "wc_table_set_launch": (ctypes.c_int, [_vp, _i32, ctypes.POINTER(WcLaunch)]),
    "wc_table_get_launch": (ctypes.c_int, [_vp, _i32, ctypes.POINTER(WcLaunch)]),
    "wc_insert": (ctypes.c_int, [_vp, _vp, _vp, _u64, _vp]),
    "wc_retrieve": (ctypes.c_int, [_vp, _vp, _u64, _vp, _vp, _vp]),
    "wc_erase": (ctypes.c_int, [_vp, _vp, _u64, _vp]),
    "wc_contains": (ctypes.c_int, [_vp, _vp, _u64, _vp, _vp]),
    "wc_insert_host": (ctypes.c_int, [_vp, _vp, _vp, _u64, _vp]),
    "wc_retrieve_host": (ctypes.c_int, [_vp, _vp, _u64, _vp, _vp, _vp]),
    "wc_count_values": (ctypes.c_int, [_vp, _vp, _u64, _vp, ctypes.POINTER(_u64), _vp]),
    "wc_retrieve_multi": (ctypes.c_int, [_vp, _vp, _u64, _vp, _vp, _vp]),
    "wc_size": (ctypes.c_int, [_vp, ctypes.POINTER(_u64), _vp]),
    "wc_num_keys": (ctypes.c_int, [_vp, ctypes.POINTER(_u64), _vp]),
    "wc_load_factor": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_double), _vp]),
    "wc_value_pool_used": (ctypes.c_int, [_vp, ctypes.POINTER(_u64), _vp]),
    "wc_get_status": (ctypes.c_int, [_vp, ctypes.POINTER(_u32), _i32, _vp]),
    "wc_check_status": (ctypes.c_int, [_vp, ctypes.POINTER(_u32), _vp]),
    "wc_table_dump_slots": (ctypes.c_int, [_vp, _vp, _u64, _vp]),
    "wc_table_device_view": (ctypes.c_int, [_vp, ctypes.POINTER(WcDeviceView)]),
    "wc_table_dump_overflow_bits": (ctypes.c_int, [_vp, _vp, _u64, _vp]),
    "wc_table_snapshot_bytes": (_u64, [_vp]),
    "wc_table_snapshot": (ctypes.c_int, [_vp, _vp, _u64, _vp]),
    "wc_table_restore": (ctypes.c_int, [_vp, _vp, _u64, _vp]),
    "wc_debug_fail_allocations": (ctypes.c_int, [_u32]),
}


def extra_signatures(sigs: dict):
    """Register further exported functions (used by the other binding modules)."""
    _SIGS.update(sigs)
    if _lib is not None:
        _bind(_lib, sigs)


def _bind(lib, sigs):
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args


def lib():
    """The loaded libwc.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libwc.so is not built (%s); build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`" % LIB_PATH)
        handle = ctypes.CDLL(LIB_PATH)
        _bind(handle, _SIGS)
        _lib = handle
    return _lib


def status_string(code: int) -> str:
    try:
        return lib().wc_status_string(int(code)).decode()
    except ImportError:
        return "status %d" % code


def check(code: int, where: str):
    if code != WC_OK:
        raise WcError(code, where)


def ptr(x) -> int | None:
    """Device address of a tensor (or an int address); None for None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, torch.Tensor):
        if x.numel() and not x.is_contiguous():
            raise ValueError("buffers must be contiguous")
        return x.data_ptr() if x.numel() else 0
    raise TypeError("expected a torch.Tensor or an integer device address, got %r" % type(x))


def stream_handle(stream) -> int | None:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream
